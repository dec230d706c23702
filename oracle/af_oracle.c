/*
 * af_oracle.c -- plain, slow, FP64 CPU oracle of one time step of the fully
 * discrete Active Flux method with transported acoustic increments (RB-TAI)
 * and of the additive Roe-Barsukow (RB) point update (arXiv 2605.12915).
 *
 * TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the CPU
 * baseline of the benchmark load this library.  It shares no code with the
 * CUDA path.  Built with -ffp-contract=off so every operation rounds once.
 *
 * Every function follows one passage of the paper and is written as the
 * passage states it -- no blocking, fusion or reordering:
 *   gas model ............................. Sec. 2 (Euler equations, EOS)
 *   centre recovery ....................... Sec. 2, Eq. (center-node); explicit
 *                                           indices in Sec. 4
 *   cellwise primitive Q2 reconstruction .. Sec. 2 (W^recon) and Sec. 4
 *                                           (Lagrange basis l_-, l_0, l_+)
 *   exact frozen acoustic operator S_ac ... Sec. 3.1 and Appendix D
 *                                           (compact monomial block)
 *   acoustic density closure .............. Sec. 3.1
 *   two-Picard convective foot ............ Eq. (adv-footpoint); Sec. 6.1 step 3
 *   RB additive point update .............. Eq. (barsukow-additive)
 *   RB-TAI transported point update ....... Eq. (transported-update); Sec. 6.1
 *                                           steps 1-4
 *   foot-centred exact acoustic update .... Appendix C, Eqs. (fc-foot-freeze),
 *                                           (fc-half-footprint),
 *                                           (fc-moment-families), (fc-role-rows)
 *   space-time Simpson flux + average ..... Sec. 3.1, Eq. (af-average-update);
 *                                           Sec. 6.1
 *   entropy functional .................... Sec. 6 (-int rho log(p/rho^gamma))
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - S_ac is applied to the raw reconstruction (not a deviation form); the
 *    increments are S_ac W - W at the node.
 *  - The frozen state of a node is the reconstruction at the node, i.e. the
 *    point value (V, E_v, E_h) or the recovered centre value (C).
 *  - RB density: rho = rho_f + (p_ac(P) - p(P)) / c_P^2 (closure of Sec. 3.1
 *    inserted in Eq. (barsukow-additive)).
 *  - Foot cell: floor of the foot position in cell units, periodic wrap.
 *  - Foot-centred update: the linear density closure of Sec. 3.1 frozen at the
 *    foot, rho = rho_* + (p - p_*)/c_*^2 (Appendix C offers it beside an
 *    isentropic one); the moments are taken by quadrature of their definition
 *    (Appendix C derives closed forms, not printed).
 */
#define _USE_MATH_DEFINES
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "af_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Gas model (Sec. 2): U = (rho, rho u, rho v, E), W = (rho, u, v, p),      */
/* E = p/(gamma-1) + rho (u^2+v^2)/2, c^2 = gamma p / rho.                  */
/* ------------------------------------------------------------------------ */
static void prim_to_cons(double gamma, const double *w, double *u) {
  u[0] = w[0];
  u[1] = w[0] * w[1];
  u[2] = w[0] * w[2];
  u[3] = w[3] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2]);
}

static void cons_to_prim(double gamma, const double *u, double *w) {
  w[0] = u[0];
  w[1] = u[1] / u[0];
  w[2] = u[2] / u[0];
  w[3] = (gamma - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]);
}

/* x-flux F(U) and y-flux G(U) of the Euler equations, from primitives */
static void flux_x(double gamma, const double *w, double *f) {
  double e = w[3] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2]);
  f[0] = w[0] * w[1];
  f[1] = w[0] * w[1] * w[1] + w[3];
  f[2] = w[0] * w[1] * w[2];
  f[3] = w[1] * (e + w[3]);
}

static void flux_y(double gamma, const double *w, double *g) {
  double e = w[3] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2]);
  g[0] = w[0] * w[2];
  g[1] = w[0] * w[1] * w[2];
  g[2] = w[0] * w[2] * w[2] + w[3];
  g[3] = w[2] * (e + w[3]);
}

/* ------------------------------------------------------------------------ */
/* Appendix D: wedge moments mu^Theta_mn = int_Theta cos^m sin^n dtheta,     */
/* zeta_j = sqrt(pi) Gamma((j+1)/2) / Gamma(j/2+1), and the 3x3 block        */
/* C^Theta_ab with input/output ordered (pi, u, v).                          */
/* ------------------------------------------------------------------------ */

/* wedge angle ranges in units of pi:
 * 0 NE [0,1/2], 1 NW [1/2,1], 2 SW [1,3/2], 3 SE [3/2,2],
 * 4 right half [-1/2,1/2], 5 left half [1/2,3/2],
 * 6 upper half [0,1], 7 lower half [1,2], 8 full disk [0,2]. */
static const double wedge_lo[9] = {0.0, 0.5, 1.0, 1.5, -0.5, 0.5, 0.0, 1.0, 0.0};
static const double wedge_hi[9] = {0.5, 1.0, 1.5, 2.0, 0.5, 1.5, 1.0, 2.0, 2.0};

static double binom(int n, int k) {
  double b = 1.0;
  for (int i = 1; i <= k; ++i) b = b * (double)(n - k + i) / (double)i;
  return b;
}

/* cos^m sin^n written as a sum of exponentials e^{i w theta}, integrated
 * exactly over [t0, t1]. */
static double wedge_moment(int m, int n, double t0, double t1) {
  double complex acc = 0.0;
  for (int k = 0; k <= m; ++k) {
    for (int l = 0; l <= n; ++l) {
      double coef = binom(m, k) * binom(n, l) * (((n - l) % 2) ? -1.0 : 1.0);
      int w = (2 * k - m) + (2 * l - n);
      double complex integral;
      if (w == 0)
        integral = t1 - t0;
      else
        integral = (cexp(I * w * t1) - cexp(I * w * t0)) / (I * (double)w);
      acc += coef * integral;
    }
  }
  acc /= pow(2.0, m) * cpow(2.0 * I, n);
  return creal(acc);
}

static double zeta(int j) {
  return sqrt(M_PI) * tgamma(0.5 * (j + 1)) / tgamma(0.5 * j + 1.0);
}

/* blk[w][a][b][out][in] */
static double blk[9][3][3][3][3];
static int blk_ready = 0;

static void compute_block(int w, int a, int b, double B[3][3]) {
  double t0 = wedge_lo[w] * M_PI, t1 = wedge_hi[w] * M_PI;
  int q = a + b;
  double chi = (q == 0) ? 1.0 : 1.0 + 1.0 / (double)q;
  double g = (double)q + 1.0 + 3.0 * chi;
  double M = wedge_moment(a, b, t0, t1) * zeta(q + 1);
  double Xm = wedge_moment(a + 2, b, t0, t1) * zeta(q + 3);
  double Ym = wedge_moment(a + 1, b + 1, t0, t1) * zeta(q + 3);
  double Zm = wedge_moment(a, b + 2, t0, t1) * zeta(q + 3);
  double Px = (q + 2) * wedge_moment(a + 1, b, t0, t1) * zeta(q + 2);
  double Py = (q + 2) * wedge_moment(a, b + 1, t0, t1) * zeta(q + 2);
  double s = 1.0 / (4.0 * M_PI);
  B[0][0] = s * (q + 1) * M;
  B[0][1] = -s * Px;
  B[0][2] = -s * Py;
  B[1][0] = -s * Px;
  B[1][1] = s * (g * Xm - chi * M);
  B[1][2] = s * g * Ym;
  B[2][0] = -s * Py;
  B[2][1] = s * g * Ym;
  B[2][2] = s * (g * Zm - chi * M);
  if (q == 0) {
    double omega = (t1 - t0) / (2.0 * M_PI);
    B[1][1] += 2.0 * omega / 3.0;
    B[2][2] += 2.0 * omega / 3.0;
  }
}

static void ensure_blocks(void) {
  if (blk_ready) return;
  for (int w = 0; w < 9; ++w)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) compute_block(w, a, b, blk[w][a][b]);
  blk_ready = 1;
}

void orc_sac_block(int w, int a, int b, double *out) {
  ensure_blocks();
  for (int o = 0; o < 3; ++o)
    for (int i = 0; i < 3; ++i) out[3 * o + i] = blk[w][a][b][o][i];
}

/* ------------------------------------------------------------------------ */
/* Cellwise Q2 Lagrange basis (Sec. 4): l_-(s) = s(s-1)/2, l_0 = 1-s^2,      */
/* l_+(s) = s(s+1)/2 on nodes s in {-1, 0, 1}.                               */
/* ------------------------------------------------------------------------ */
static void lagrange3(double s, double l[3]) {
  l[0] = 0.5 * s * (s - 1.0);
  l[1] = 1.0 - s * s;
  l[2] = 0.5 * s * (s + 1.0);
}

/* Coefficients (powers X^0, X^1, X^2) of l_m(alpha + beta X), obtained by
 * multiplying the two linear factors of the Lagrange polynomial. */
static void lagrange3_poly(int m, double alpha, double beta, double c[3]) {
  static const double nodes[3] = {-1.0, 0.0, 1.0};
  c[0] = 1.0;
  c[1] = 0.0;
  c[2] = 0.0;
  for (int k = 0; k < 3; ++k) {
    if (k == m) continue;
    double d = nodes[m] - nodes[k];
    double a0 = (alpha - nodes[k]) / d, a1 = beta / d; /* factor a0 + a1 X */
    double n0 = c[0] * a0;
    double n1 = c[1] * a0 + c[0] * a1;
    double n2 = c[2] * a0 + c[1] * a1;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
  }
}

/* Monomial coefficients mono[a][b] of X^a Y^b of the Q2 polynomial with
 * nodal values f[ix][iy], in coordinates X = (x - x_K)/h, Y = (y - y_K)/h
 * centred at a node located at (ox, oy) cell units from the cell's lower-left
 * corner.  Cell local coordinate xi = 2((x - x_i)/h) - 1 = (2 ox - 1) + 2 X. */
static void q2_to_monomials(const double f[3][3], double ox, double oy, double mono[3][3]) {
  double lx[3][3], ly[3][3];
  for (int m = 0; m < 3; ++m) {
    lagrange3_poly(m, 2.0 * ox - 1.0, 2.0, lx[m]);
    lagrange3_poly(m, 2.0 * oy - 1.0, 2.0, ly[m]);
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) s += f[m][n] * lx[m][a] * ly[n][b];
      mono[a][b] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Node families and their wedges (Sec. 3.1: a vertex uses four quadrant     */
/* wedges, an edge midpoint two half planes, the cell centre the full disk). */
/* ------------------------------------------------------------------------ */
typedef struct {
  int nw;          /* number of wedges */
  int wedge[4];    /* wedge id (see wedge_lo / wedge_hi) */
  int di[4], dj[4];/* adjacent cell relative to the node's owner cell (i,j) */
  double ox[4], oy[4]; /* node position inside that cell, cell units */
  double px, py;   /* node position relative to (x_i, y_j), cell units */
} family_t;

static const family_t families[4] = {
    /* V(i,j) at (x_i, y_j): NE = C_ij, NW = C_{i-1,j}, SW = C_{i-1,j-1}, SE = C_{i,j-1} */
    {4, {0, 1, 2, 3}, {0, -1, -1, 0}, {0, 0, -1, -1}, {0.0, 1.0, 1.0, 0.0}, {0.0, 0.0, 1.0, 1.0}, 0.0, 0.0},
    /* E_v(i,j) at (x_i, y_{j+1/2}): right = C_ij, left = C_{i-1,j} */
    {2, {4, 5, 0, 0}, {0, -1, 0, 0}, {0, 0, 0, 0}, {0.0, 1.0, 0, 0}, {0.5, 0.5, 0, 0}, 0.0, 0.5},
    /* E_h(i,j) at (x_{i+1/2}, y_j): upper = C_ij, lower = C_{i,j-1} */
    {2, {6, 7, 0, 0}, {0, 0, 0, 0}, {0, -1, 0, 0}, {0.5, 0.5, 0, 0}, {0.0, 1.0, 0, 0}, 0.5, 0.0},
    /* C(i,j) at (x_{i+1/2}, y_{j+1/2}): full disk of C_ij */
    {1, {8, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0.5, 0, 0, 0}, {0.5, 0, 0, 0}, 0.5, 0.5},
};

/* Exact frozen acoustic evolution at one node (Sec. 3.1, Appendix D): the
 * local data of each wedge is the adjacent cell's Q2 polynomial of
 * (pi = p/Z, u, v); out(pi,u,v) = sum_wedges sum_ab r^{a+b} C^Theta_ab coef_ab. */
void orc_sac_node(int fam, const double *cells, double r, double Z, double *out) {
  ensure_blocks();
  const family_t *F = &families[fam];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < F->nw; ++k) {
    const double *c = cells + 27 * k;
    double fp[3][3], fu[3][3], fv[3][3];
    for (int ix = 0; ix < 3; ++ix)
      for (int iy = 0; iy < 3; ++iy) {
        fp[ix][iy] = c[0 + 3 * ix + iy] / Z; /* pi = p / (rho_0 c_0) */
        fu[ix][iy] = c[9 + 3 * ix + iy];
        fv[ix][iy] = c[18 + 3 * ix + iy];
      }
    double mono[3][3][3];
    q2_to_monomials(fp, F->ox[k], F->oy[k], mono[0]);
    q2_to_monomials(fu, F->ox[k], F->oy[k], mono[1]);
    q2_to_monomials(fv, F->ox[k], F->oy[k], mono[2]);
    int w = F->wedge[k];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double rq = pow(r, a + b);
        for (int o = 0; o < 3; ++o)
          for (int in = 0; in < 3; ++in) acc[o] += rq * blk[w][a][b][o][in] * mono[in][a][b];
      }
  }
  out[0] = Z * acc[0]; /* p_ac = Z pi_ac */
  out[1] = acc[1];
  out[2] = acc[2];
}

/* ------------------------------------------------------------------------ */
/* Grid access (Sec. 2): periodic Cartesian grid.                            */
/* ------------------------------------------------------------------------ */
static int wrap(int i, int n) { return ((i % n) + n) % n; }

#define AVG(st, N, k) ((st) + (size_t)(k) * (N))
#define VTX(st, N, k) ((st) + (size_t)(4 + (k)) * (N))
#define EVP(st, N, k) ((st) + (size_t)(8 + (k)) * (N))
#define EHP(st, N, k) ((st) + (size_t)(12 + (k)) * (N))

/* primitive point value of a family at integer position (wrapped) */
static void point_value(int nx, int ny, const double *st, int fam, int i, int j, double w[4]) {
  size_t N = (size_t)nx * ny;
  size_t id = (size_t)wrap(j, ny) * nx + wrap(i, nx);
  int base = (fam == ORC_NODE_V) ? 4 : (fam == ORC_NODE_EV) ? 8 : 12;
  for (int k = 0; k < 4; ++k) w[k] = st[(size_t)(base + k) * N + id];
}

/* primitive value of a family from a block of 12 point planes (V, E_v, E_h) */
static void level_value(int nx, int ny, const double *pts, int fam, int i, int j, double w[4]) {
  size_t N = (size_t)nx * ny;
  size_t id = (size_t)wrap(j, ny) * nx + wrap(i, nx);
  for (int k = 0; k < 4; ++k) w[k] = pts[(size_t)(4 * fam + k) * N + id];
}

/* the nine primitive nodal values of cell C_ij, f[ix][iy][field] with
 * xi, eta = -1, 0, 1 (Sec. 4, nodal placement of R_Delta). */
static void cell_nodes(int nx, int ny, const double *st, const double *wc, int i, int j,
                       double f[3][3][4]) {
  size_t N = (size_t)nx * ny;
  point_value(nx, ny, st, ORC_NODE_V, i, j, f[0][0]);
  point_value(nx, ny, st, ORC_NODE_EH, i, j, f[1][0]);
  point_value(nx, ny, st, ORC_NODE_V, i + 1, j, f[2][0]);
  point_value(nx, ny, st, ORC_NODE_EV, i, j, f[0][1]);
  size_t id = (size_t)wrap(j, ny) * nx + wrap(i, nx);
  for (int k = 0; k < 4; ++k) f[1][1][k] = wc[(size_t)k * N + id];
  point_value(nx, ny, st, ORC_NODE_EV, i + 1, j, f[2][1]);
  point_value(nx, ny, st, ORC_NODE_V, i, j + 1, f[0][2]);
  point_value(nx, ny, st, ORC_NODE_EH, i, j + 1, f[1][2]);
  point_value(nx, ny, st, ORC_NODE_V, i + 1, j + 1, f[2][2]);
}

/* ------------------------------------------------------------------------ */
/* Centre recovery by inverting the tensor Simpson rule in conservative      */
/* variables (Sec. 2, Eq. center-node; explicit indices in Sec. 4).          */
/* ------------------------------------------------------------------------ */
int orc_center_recovery(int nx, int ny, double gamma, const double *st, double *wc) {
  size_t N = (size_t)nx * ny;
  int flags = 0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double w[4], u[4], ubar[4], corners[4] = {0, 0, 0, 0}, edges[4] = {0, 0, 0, 0};
      size_t id = (size_t)j * nx + i;
      for (int k = 0; k < 4; ++k) ubar[k] = AVG(st, N, k)[id];
      const int cfam[4] = {ORC_NODE_V, ORC_NODE_V, ORC_NODE_V, ORC_NODE_V};
      const int ci[4] = {i, i + 1, i, i + 1}, cj[4] = {j, j, j + 1, j + 1};
      for (int c = 0; c < 4; ++c) {
        point_value(nx, ny, st, cfam[c], ci[c], cj[c], w);
        prim_to_cons(gamma, w, u);
        for (int k = 0; k < 4; ++k) corners[k] += u[k];
      }
      const int efam[4] = {ORC_NODE_EH, ORC_NODE_EH, ORC_NODE_EV, ORC_NODE_EV};
      const int ei[4] = {i, i, i, i + 1}, ej[4] = {j, j + 1, j, j};
      for (int c = 0; c < 4; ++c) {
        point_value(nx, ny, st, efam[c], ei[c], ej[c], w);
        prim_to_cons(gamma, w, u);
        for (int k = 0; k < 4; ++k) edges[k] += u[k];
      }
      double uc[4], wcv[4];
      for (int k = 0; k < 4; ++k)
        uc[k] = 9.0 / 4.0 * (ubar[k] - corners[k] / 36.0 - edges[k] / 9.0);
      cons_to_prim(gamma, uc, wcv);
      if (!(wcv[0] > 0.0) || !(wcv[3] > 0.0)) flags |= ORC_FLAG_NONPHYSICAL;
      for (int k = 0; k < 4; ++k) wc[(size_t)k * N + id] = wcv[k];
    }
  return flags;
}

/* ------------------------------------------------------------------------ */
/* Evaluation of a cellwise Q2 field at a point in cell units (Sec. 4 and    */
/* Eq. reconstruction-row: r = floor(x), s = floor(y), periodic wrap).       */
/* ------------------------------------------------------------------------ */
static void locate(double X, double Y, int *ci, int *cj, double *xi, double *eta) {
  double fx = floor(X), fy = floor(Y);
  *ci = (int)fx;
  *cj = (int)fy;
  *xi = 2.0 * (X - fx - 0.5);
  *eta = 2.0 * (Y - fy - 0.5);
}

void orc_recon_eval(int nx, int ny, const double *st, const double *wc, double X, double Y,
                    double *out) {
  int ci, cj;
  double xi, eta, lx[3], ly[3], f[3][3][4];
  locate(X, Y, &ci, &cj, &xi, &eta);
  cell_nodes(nx, ny, st, wc, ci, cj, f);
  lagrange3(xi, lx);
  lagrange3(eta, ly);
  for (int k = 0; k < 4; ++k) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) s += lx[a] * ly[b] * f[a][b][k];
    out[k] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Frozen state of a node (Sec. 6.1 step 1): W_K = R_h W(X_K), i.e. the     */
/* point value, or the recovered centre for the C family.                    */
/* ------------------------------------------------------------------------ */
static void node_state(int nx, int ny, const double *st, const double *wc, int fam, int i,
                       int j, double w[4]) {
  if (fam == ORC_NODE_C) {
    size_t N = (size_t)nx * ny;
    size_t id = (size_t)wrap(j, ny) * nx + wrap(i, nx);
    for (int k = 0; k < 4; ++k) w[k] = wc[(size_t)k * N + id];
  } else {
    point_value(nx, ny, st, fam, i, j, w);
  }
}

/* Acoustic outputs (p_ac, u_ac, v_ac) at every node of a family, duration tau
 * (Sec. 6.1 step 1; Sec. 3.1).  ac holds 3*N doubles: u_ac, v_ac, p_ac planes. */
static int acoustic_outputs(int nx, int ny, double h, double gamma, double tau, int fam,
                            const double *st, const double *wc, double *ac) {
  size_t N = (size_t)nx * ny;
  const family_t *F = &families[fam];
  int flags = 0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double wk[4];
      node_state(nx, ny, st, wc, fam, i, j, wk);
      if (!(wk[0] > 0.0) || !(wk[3] > 0.0)) flags |= ORC_FLAG_NONPHYSICAL;
      double c = sqrt(gamma * wk[3] / wk[0]);
      double Z = wk[0] * c;
      double r = c * tau / h;
      double cells[4 * 27];
      for (int k = 0; k < F->nw; ++k) {
        double f[3][3][4];
        cell_nodes(nx, ny, st, wc, i + F->di[k], j + F->dj[k], f);
        for (int ix = 0; ix < 3; ++ix)
          for (int iy = 0; iy < 3; ++iy) {
            cells[27 * k + 0 + 3 * ix + iy] = f[ix][iy][3];
            cells[27 * k + 9 + 3 * ix + iy] = f[ix][iy][1];
            cells[27 * k + 18 + 3 * ix + iy] = f[ix][iy][2];
          }
      }
      double out[3];
      orc_sac_node(fam, cells, r, Z, out);
      size_t id = (size_t)j * nx + i;
      ac[0 * N + id] = out[1];
      ac[1 * N + id] = out[2];
      ac[2 * N + id] = out[0];
    }
  return flags;
}

int orc_acoustic_increments(int nx, int ny, double h, double gamma, double tau, int fam,
                            const double *st, const double *wc, double *d) {
  size_t N = (size_t)nx * ny;
  int flags = acoustic_outputs(nx, ny, h, gamma, tau, fam, st, wc, d);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double wk[4];
      node_state(nx, ny, st, wc, fam, i, j, wk);
      size_t id = (size_t)j * nx + i;
      d[0 * N + id] -= wk[1]; /* Delta u */
      d[1 * N + id] -= wk[2]; /* Delta v */
      d[2 * N + id] -= wk[3]; /* Delta p */
    }
  return flags;
}

/* Q2 interpolant I_h Delta of the nodal increments in the cell containing a
 * point (Sec. 4, R_Delta; Sec. 6.1 step 2).  dfam[fam] = 3 planes (du,dv,dp). */
static void increment_eval(int nx, int ny, double *const dfam[4], double X, double Y,
                           double out[3]) {
  size_t N = (size_t)nx * ny;
  int ci, cj;
  double xi, eta, lx[3], ly[3];
  locate(X, Y, &ci, &cj, &xi, &eta);
  lagrange3(xi, lx);
  lagrange3(eta, ly);
  /* nodal placement: [ix][iy] -> family and integer position */
  const int nfam[3][3] = {{ORC_NODE_V, ORC_NODE_EV, ORC_NODE_V},
                          {ORC_NODE_EH, ORC_NODE_C, ORC_NODE_EH},
                          {ORC_NODE_V, ORC_NODE_EV, ORC_NODE_V}};
  const int ndi[3][3] = {{0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
  const int ndj[3][3] = {{0, 0, 1}, {0, 0, 1}, {0, 0, 1}};
  for (int k = 0; k < 3; ++k) out[k] = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      size_t id = (size_t)wrap(cj + ndj[a][b], ny) * nx + wrap(ci + ndi[a][b], nx);
      const double *d = dfam[nfam[a][b]];
      for (int k = 0; k < 3; ++k) out[k] += lx[a] * ly[b] * d[(size_t)k * N + id];
    }
}

/* ------------------------------------------------------------------------ */
/* Foot-centred exact frozen acoustic update (Appendix C).  The acoustic    */
/* disk of radius R = c_* tau is centred at the convective foot F (not at a */
/* node); the frozen state is the reconstruction at F (Eq. fc-foot-freeze). */
/* Under the compact footprint condition (Eq. fc-half-footprint) the disk   */
/* lies in the cells around the target point and is cut only by the grid   */
/* lines through that point: a vertex disk into up to four fragments, an    */
/* edge disk into up to two.                                                 */
/*                                                                           */
/* The exact solution of frozen linear acoustics u_t + c grad pi = 0,        */
/* pi_t + c div u = 0 at the centre of the disk, written with the projected-*/
/* sphere mean S[f](R) = (1/4pi) int_{B1} f(F + R w) Psi(w) dw,              */
/* Psi = 2 (1 - |w|^2)^{-1/2} (the 2D Poisson formula by descent):           */
/*   pi(F, tau) = d/dR [R S[pi_0](R)] - R S[div u_0](R)                      */
/*   u(F, tau)  = u_0(F) - R S[grad pi_0](R) + R G(R) + int_0^R G(s) ds,     */
/*   G_j(s) = (1/4pi) int_{B1} (w_1 d_j u_0 + w_2 d_j v_0)(F + s w) Psi dw,  */
/* where the second line follows from u_t = -c grad pi, the divergence     */
/* theorem on the ball of radius s in the z-extended 3D problem, and one    */
/* integration by parts in s.  For continuous piecewise-Q2 data every term  */
/* is a sum over fragments of the fragment's polynomial (in monomials about */
/* F) against the fragment's moments m_ij(R) = int xi^i eta^j Psi over the  */
/* fragment scaled to the unit disk, their radius derivative and their      */
/* history integral (Eq. fc-moment-families).  On a node-centred disk the   */
/* fragments are the wedges of Sec. 3.1 and the sum equals the Appendix D   */
/* update.  Here the moments are computed by direct quadrature: for every   */
/* ray from F the radial integrals are closed forms, and the angular        */
/* integral is taken by tanh-sinh quadrature between the angles at which    */
/* the ray's clipping changes form.  Lengths are in units of h.             */
/* ------------------------------------------------------------------------ */

/* int_0^phi sin^k t dt */
static double sin_power_integral(int k, double phi) {
  if (k == 0) return phi;
  if (k == 1) return 1.0 - cos(phi);
  return -pow(sin(phi), k - 1) * cos(phi) / k + (double)(k - 1) / k * sin_power_integral(k - 2, phi);
}

/* One fragment: the points x (offsets from F, units of h) with
 * sgn[c] * (x[axis[c]] - d[c]) >= 0 for its n constraints. */
typedef struct {
  int n;
  int axis[2];
  double sgn[2], d[2];
} fc_frag_t;

/* the part [lo, hi] of the ray from F at angle th inside the fragment and the
 * disk of radius r; 0 if empty */
static int fc_ray(const fc_frag_t *g, double r, double th, double *lo, double *hi) {
  double a = 0.0, b = r;
  double e[2] = {cos(th), sin(th)};
  for (int c = 0; c < g->n; ++c) {
    double se = g->sgn[c] * e[g->axis[c]];
    if (se == 0.0) {
      if (-g->sgn[c] * g->d[c] < 0.0) return 0;
      continue;
    }
    double t = g->d[c] / e[g->axis[c]];
    if (se > 0.0) {
      if (t > a) a = t;
    } else if (t < b) {
      b = t;
    }
  }
  if (!(a < b)) return 0;
  *lo = a;
  *hi = b;
  return 1;
}

/* moment arrays of one fragment of the disk of radius r (units of h):
 *   m[i][j] = int xi^i eta^j Psi over the fragment scaled to the unit disk,
 *   E[a][b] = r^-q d/dr (r^{q+1} m_ab(r)), q = a + b,
 *   H[i][j] = int_0^r s^{i+j-1} m_ij(s) ds (i + j >= 1).
 * On a ray the fragment is lo <= rho <= hi; with rho = r sin(phi) the radial
 * parts are sin-power integrals. */
static void fc_ray_terms(double r, double th, double lo, double hi, int hi_on_circle,
                         double m[5][5], double E[3][3], double H[5][5]) {
  double plo = asin(fmin(lo / r, 1.0));
  double phi_hi = hi_on_circle ? 0.5 * M_PI : asin(fmin(hi / r, 1.0));
  double K_lo[7], K_hi[7];
  for (int k = 0; k < 7; ++k) {
    K_lo[k] = sin_power_integral(k, plo);
    K_hi[k] = sin_power_integral(k, phi_hi);
  }
  double c = cos(th), s = sin(th);
  double cp[5], sp[5];
  cp[0] = sp[0] = 1.0;
  for (int k = 1; k < 5; ++k) {
    cp[k] = cp[k - 1] * c;
    sp[k] = sp[k - 1] * s;
  }
  /* d/dr of r^k K_k(asin(x/r)) = r^{k-1} [k K_k(phi) - sin^k(phi) tan(phi)] */
  double tan_lo = lo > 0.0 ? (lo / r) / sqrt(fmax(1.0 - (lo / r) * (lo / r), 0.0)) : 0.0;
  double tan_hi = hi_on_circle ? 0.0 : (hi / r) / sqrt(fmax(1.0 - (hi / r) * (hi / r), 0.0));
  for (int i = 0; i < 5; ++i)
    for (int j = 0; i + j < 5; ++j) {
      int k = i + j + 1;
      double ang = cp[i] * sp[j];
      m[i][j] = 2.0 * ang * (K_hi[k] - K_lo[k]);
      if (i + j >= 1) {
        int q = i + j;
        double L_hi = K_hi[q - 1] - K_hi[q + 1], L_lo = K_lo[q - 1] - K_lo[q + 1];
        H[i][j] = 2.0 * pow(r, q) * ang * (L_hi - L_lo);
      } else {
        H[i][j] = 0.0;
      }
      if (i < 3 && j < 3) {
        double v = k * K_hi[k] - k * K_lo[k] + pow(lo / r, k) * tan_lo;
        if (!hi_on_circle) v -= pow(hi / r, k) * tan_hi;
        E[i][j] = 2.0 * ang * v;
      }
    }
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return x < y ? -1 : x > y;
}

static void fc_fragment_moments(const fc_frag_t *g, double r, double m[5][5], double E[3][3],
                                double H[5][5]) {
  memset(m, 0, sizeof(double) * 25);
  memset(E, 0, sizeof(double) * 9);
  memset(H, 0, sizeof(double) * 25);
  /* angles where the ray's clipping changes form */
  double br[16];
  int nb = 0;
  for (int k = 0; k <= 4; ++k) br[nb++] = 0.5 * M_PI * k;
  for (int c = 0; c < g->n; ++c) {
    double d = g->d[c];
    if (fabs(d) < r) {
      double a = g->axis[c] == 0 ? acos(d / r) : asin(d / r);
      double a2 = g->axis[c] == 0 ? 2.0 * M_PI - a : M_PI - a;
      br[nb++] = fmod(a + 2.0 * M_PI, 2.0 * M_PI);
      br[nb++] = fmod(a2 + 2.0 * M_PI, 2.0 * M_PI);
    }
  }
  if (g->n == 2 && g->axis[0] != g->axis[1]) {
    double dx = g->axis[0] == 0 ? g->d[0] : g->d[1], dy = g->axis[0] == 0 ? g->d[1] : g->d[0];
    br[nb++] = fmod(atan2(dy, dx) + 2.0 * M_PI, 2.0 * M_PI);
  }
  qsort(br, nb, sizeof(double), cmp_double);
  /* tanh-sinh rule on each piece: t = k/16, |k| <= 64 */
  const double hstep = 1.0 / 16.0;
  for (int p = 0; p + 1 < nb; ++p) {
    double a = br[p], b = br[p + 1];
    if (!(b - a > 1e-14)) continue;
    double mid = 0.5 * (a + b), half = 0.5 * (b - a);
    for (int k = -64; k <= 64; ++k) {
      double t = k * hstep;
      double u = 0.5 * M_PI * sinh(t);
      double x = tanh(u), w = hstep * 0.5 * M_PI * cosh(t) / (cosh(u) * cosh(u));
      if (w < 1e-300) continue;
      double th = mid + half * x, lo, hi;
      if (!fc_ray(g, r, th, &lo, &hi)) continue;
      double mm[5][5], ee[3][3], hh[5][5];
      fc_ray_terms(r, th, lo, hi, hi >= r, mm, ee, hh);
      double ww = half * w;
      for (int i = 0; i < 5; ++i)
        for (int j = 0; i + j < 5; ++j) {
          m[i][j] += ww * mm[i][j];
          H[i][j] += ww * hh[i][j];
          if (i < 3 && j < 3) E[i][j] += ww * ee[i][j];
        }
    }
  }
}

/* Exact frozen acoustic evolution at the centre F of a disk of radius r (units
 * of h) from fragments of continuous piecewise-Q2 data.  mono[f][k][a][b] is the
 * polynomial of fragment f, field k = (pi, u, v), in monomials X^a Y^b about F
 * (units of h).  out = (pi, u, v) at F after the evolution. */
static void fc_evolve(int nf, const fc_frag_t *frags, double mono[][3][3][3], double r,
                      double out[3]) {
  double pi_out = 0.0, du = 0.0, dv = 0.0;
  /* u_0(F): the constant coefficient of the fragment whose cell holds F (every
   * constraint holds at the centre; on a grid line either side's polynomial
   * gives the same value, the data being continuous) */
  double u0 = 0.0, v0 = 0.0;
  for (int f = 0; f < nf; ++f) {
    int holds = 1;
    for (int c = 0; c < frags[f].n; ++c)
      if (frags[f].sgn[c] * (0.0 - frags[f].d[c]) < 0.0) holds = 0;
    if (holds) {
      u0 = mono[f][1][0][0];
      v0 = mono[f][2][0][0];
      break;
    }
  }
  for (int f = 0; f < nf; ++f) {
    double m[5][5], E[3][3], H[5][5];
    fc_fragment_moments(&frags[f], r, m, E, H);
    double(*P)[3] = mono[f][0];
    double(*U)[3] = mono[f][1];
    double(*V)[3] = mono[f][2];
#define MM(i, j) (((i) < 0 || (j) < 0) ? 0.0 : m[i][j])
#define HH(i, j) (((i) < 0 || (j) < 0) ? 0.0 : H[i][j])
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        int q = a + b;
        double rq = pow(r, q);
        /* pi: d/dR [R S[pi_0]] - R S[div u_0] */
        pi_out += rq * (P[a][b] * E[a][b] - a * U[a][b] * MM(a - 1, b) - b * V[a][b] * MM(a, b - 1));
        /* velocity: - R S[grad pi_0] + R G(R) + int_0^R G */
        du += rq * (-a * P[a][b] * MM(a - 1, b) + a * U[a][b] * MM(a, b) +
                    a * V[a][b] * MM(a - 1, b + 1));
        dv += rq * (-b * P[a][b] * MM(a, b - 1) + b * U[a][b] * MM(a + 1, b - 1) +
                    b * V[a][b] * MM(a, b));
        if (q >= 1) {
          du += a * U[a][b] * HH(a, b) + a * V[a][b] * HH(a - 1, b + 1);
          dv += b * U[a][b] * HH(a + 1, b - 1) + b * V[a][b] * HH(a, b);
        }
      }
#undef MM
#undef HH
  }
  out[0] = pi_out / (4.0 * M_PI);
  out[1] = u0 + du / (4.0 * M_PI);
  out[2] = v0 + dv / (4.0 * M_PI);
}

/* The fragments of the disk around a point of family fam whose grid lines lie
 * at offsets (dX, dY) from F (units of h), in the cell order of `families`
 * (V: NE, NW, SW, SE; E_v: right, left; E_h: upper, lower). */
static int fc_fragments(int fam, double dX, double dY, fc_frag_t *g) {
  static const double sx[4] = {1.0, -1.0, -1.0, 1.0}, sy[4] = {1.0, 1.0, -1.0, -1.0};
  if (fam == ORC_NODE_V) {
    for (int k = 0; k < 4; ++k) {
      g[k].n = 2;
      g[k].axis[0] = 0;
      g[k].sgn[0] = sx[k];
      g[k].d[0] = dX;
      g[k].axis[1] = 1;
      g[k].sgn[1] = sy[k];
      g[k].d[1] = dY;
    }
    return 4;
  }
  for (int k = 0; k < 2; ++k) {
    g[k].n = 1;
    g[k].axis[0] = fam == ORC_NODE_EV ? 0 : 1;
    g[k].sgn[0] = k == 0 ? 1.0 : -1.0;
    g[k].d[0] = fam == ORC_NODE_EV ? dX : dY;
  }
  return 2;
}

/* Test hook: the foot-centred evolution for given cell data.  cells as in
 * orc_sac_node (raw p, u, v nodal values of each adjacent cell of the family,
 * in the family's cell order); (fx, fy) = F - P in units of h; r = c_* tau / h;
 * Z = rho_* c_*.  out = (p, u, v) at F. */
void orc_fc_node(int fam, const double *cells, double fx, double fy, double r, double Z,
                 double *out) {
  const family_t *F = &families[fam];
  fc_frag_t g[4];
  int nf = fc_fragments(fam, -fx, -fy, g);
  double mono[4][3][3][3];
  for (int k = 0; k < nf; ++k)
    for (int fld = 0; fld < 3; ++fld) {
      double f[3][3];
      for (int ix = 0; ix < 3; ++ix)
        for (int iy = 0; iy < 3; ++iy)
          f[ix][iy] = cells[27 * k + 9 * fld + 3 * ix + iy] / (fld == 0 ? Z : 1.0);
      q2_to_monomials(f, F->ox[k] + fx, F->oy[k] + fy, mono[k][fld]);
    }
  double o[3];
  fc_evolve(nf, g, mono, r, o);
  out[0] = Z * o[0];
  out[1] = o[1];
  out[2] = o[2];
}

/* Foot-centred point value (Appendix C) of family fam at (i, j) for duration
 * tau, the foot at (Xf, Yf) cell units with reconstruction wf = W_h(F).  The
 * density follows the acoustic closure of Sec. 3.1 frozen at F,
 * rho = rho_* + (p - p_*) / c_*^2.  Returns ORC_FLAG_CFL if the compact
 * footprint condition |F - P|_x + R < h/2, |F - P|_y + R < h/2 fails. */
static int fc_point(int nx, int ny, double h, double gamma, double tau, int fam, int i, int j,
                    const double *st, const double *wc, double Xf, double Yf,
                    const double wf[4], double nw[4]) {
  const family_t *F = &families[fam];
  int flags = 0;
  if (!(wf[0] > 0.0) || !(wf[3] > 0.0)) flags |= ORC_FLAG_NONPHYSICAL;
  double cs = sqrt(gamma * wf[3] / wf[0]);
  double Z = wf[0] * cs;
  double r = cs * tau / h;
  double X = i + F->px, Y = j + F->py;
  double fx = Xf - X, fy = Yf - Y; /* F - P, units of h */
  if (!(fabs(fx) + r < 0.5) || !(fabs(fy) + r < 0.5)) flags |= ORC_FLAG_CFL;
  double cells[4 * 27];
  for (int k = 0; k < F->nw; ++k) {
    double f[3][3][4];
    cell_nodes(nx, ny, st, wc, i + F->di[k], j + F->dj[k], f);
    for (int ix = 0; ix < 3; ++ix)
      for (int iy = 0; iy < 3; ++iy) {
        cells[27 * k + 0 + 3 * ix + iy] = f[ix][iy][3];
        cells[27 * k + 9 + 3 * ix + iy] = f[ix][iy][1];
        cells[27 * k + 18 + 3 * ix + iy] = f[ix][iy][2];
      }
  }
  double out[3];
  orc_fc_node(fam, cells, fx, fy, r, Z, out);
  nw[3] = out[0];
  nw[1] = out[1];
  nw[2] = out[2];
  nw[0] = wf[0] + (out[0] - wf[3]) / (cs * cs);
  return flags;
}

/* ------------------------------------------------------------------------ */
/* Point update at tau (Sec. 6.1 steps 3-4; Eq. adv-footpoint;               */
/* Eq. barsukow-additive for RB).  Writes the four new planes of a family.   */
/* ------------------------------------------------------------------------ */
static int point_update(int nx, int ny, double h, double gamma, double tau, int fam,
                        int variant, const double *st, const double *wc,
                        double *const dfam[4], const double *ac_fam, double *outw) {
  size_t N = (size_t)nx * ny;
  const family_t *F = &families[fam];
  int flags = 0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t id = (size_t)j * nx + i;
      double X = i + F->px, Y = j + F->py;
      /* two-Picard convective foot, velocities from R_h^n W only */
      double wp[4], w1[4], wf[4];
      orc_recon_eval(nx, ny, st, wc, X, Y, wp);
      double X1 = X - tau * wp[1] / h, Y1 = Y - tau * wp[2] / h;
      orc_recon_eval(nx, ny, st, wc, X1, Y1, w1);
      double Xf = X - tau * w1[1] / h, Yf = Y - tau * w1[2] / h;
      orc_recon_eval(nx, ny, st, wc, Xf, Yf, wf);
      double nw[4];
      if (variant == ORC_FC) {
        flags |= fc_point(nx, ny, h, gamma, tau, fam, i, j, st, wc, Xf, Yf, wf, nw);
      } else if (variant == ORC_TAI) {
        double d[3];
        increment_eval(nx, ny, dfam, Xf, Yf, d);
        if (!(wf[0] > 0.0) || !(wf[3] > 0.0)) flags |= ORC_FLAG_NONPHYSICAL;
        double cf2 = gamma * wf[3] / wf[0];
        nw[0] = wf[0] + d[2] / cf2;
        nw[1] = wf[1] + d[0];
        nw[2] = wf[2] + d[1];
        nw[3] = wf[3] + d[2];
      } else {
        double wk[4];
        point_value(nx, ny, st, fam, i, j, wk);
        double uac = ac_fam[0 * N + id], vac = ac_fam[1 * N + id], pac = ac_fam[2 * N + id];
        double cp2 = gamma * wk[3] / wk[0];
        double rhoac = wk[0] + (pac - wk[3]) / cp2;
        nw[0] = rhoac + wf[0] - wk[0];
        nw[1] = uac + wf[1] - wk[1];
        nw[2] = vac + wf[2] - wk[2];
        nw[3] = pac + wf[3] - wk[3];
      }
      for (int k = 0; k < 4; ++k) outw[(size_t)k * N + id] = nw[k];
    }
  return flags;
}

/* ------------------------------------------------------------------------ */
/* One full step (Sec. 6.1, Algorithm; Eq. af-average-update).               */
/* ------------------------------------------------------------------------ */
int orc_step(int nx, int ny, double h, double gamma, double dt, int variant, const double *in,
             double *out) {
  size_t N = (size_t)nx * ny;
  int flags = 0;
  double *wc = (double *)malloc(sizeof(double) * 4 * N);
  double *ac = (double *)malloc(sizeof(double) * 3 * 4 * N);  /* per family */
  double *dd = (double *)malloc(sizeof(double) * 3 * 4 * N);  /* per family */
  double *half = (double *)malloc(sizeof(double) * 12 * N);   /* V,Ev,Eh at n+1/2 */
  double *full = out + 4 * N;                                 /* V,Ev,Eh at n+1 */

  flags |= orc_center_recovery(nx, ny, gamma, in, wc);

  /* acoustic CFL at every node: c_K dt / h <= 1/2 (Sec. 3.1, Sec. 6); the
   * foot-centred update checks its own footprint condition instead */
  for (int fam = 0; fam < 4 && variant != ORC_FC; ++fam)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double wk[4];
        node_state(nx, ny, in, wc, fam, i, j, wk);
        if (wk[0] > 0.0 && wk[3] > 0.0 && sqrt(gamma * wk[3] / wk[0]) * dt / h > 0.5)
          flags |= ORC_FLAG_CFL;
      }

  const double taus[2] = {0.5 * dt, dt};
  for (int s = 0; s < 2; ++s) {
    double tau = taus[s];
    double *dfam[4];
    for (int fam = 0; fam < 4; ++fam) {
      double *acf = ac + (size_t)fam * 3 * N;
      dfam[fam] = dd + (size_t)fam * 3 * N;
      if (variant == ORC_FC) continue; /* no nodal increments: the disk sits at the foot */
      flags |= acoustic_outputs(nx, ny, h, gamma, tau, fam, in, wc, acf);
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          double wk[4];
          node_state(nx, ny, in, wc, fam, i, j, wk);
          size_t id = (size_t)j * nx + i;
          dfam[fam][0 * N + id] = acf[0 * N + id] - wk[1];
          dfam[fam][1 * N + id] = acf[1 * N + id] - wk[2];
          dfam[fam][2 * N + id] = acf[2 * N + id] - wk[3];
        }
    }
    double *dst = (s == 0) ? half : full;
    for (int fam = 0; fam < 3; ++fam)
      flags |= point_update(nx, ny, h, gamma, tau, fam, variant, in, wc, dfam,
                            ac + (size_t)fam * 3 * N, dst + (size_t)fam * 4 * N);
  }

  /* space-time Simpson fluxes and conservative average update */
  const double *lev[3] = {in + 4 * N, half, full}; /* V,Ev,Eh planes at sigma = 0, 1/2, 1 */
  const double tw[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
  double *fx = (double *)malloc(sizeof(double) * 4 * N);
  double *gy = (double *)malloc(sizeof(double) * 4 * N);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t id = (size_t)j * nx + i;
      double fhat[4] = {0, 0, 0, 0}, ghat[4] = {0, 0, 0, 0};
      for (int s = 0; s < 3; ++s) {
        double wa[4], wb[4], wm[4], fa[4], fb[4], fm[4];
        /* vertical edge x = x_i: V(i,j), E_v(i,j), V(i,j+1) */
        level_value(nx, ny, lev[s], ORC_NODE_V, i, j, wa);
        level_value(nx, ny, lev[s], ORC_NODE_EV, i, j, wm);
        level_value(nx, ny, lev[s], ORC_NODE_V, i, j + 1, wb);
        flux_x(gamma, wa, fa);
        flux_x(gamma, wm, fm);
        flux_x(gamma, wb, fb);
        for (int k = 0; k < 4; ++k) fhat[k] += tw[s] * (fa[k] + 4.0 * fm[k] + fb[k]) / 6.0;
        /* horizontal edge y = y_j: V(i,j), E_h(i,j), V(i+1,j) */
        level_value(nx, ny, lev[s], ORC_NODE_V, i, j, wa);
        level_value(nx, ny, lev[s], ORC_NODE_EH, i, j, wm);
        level_value(nx, ny, lev[s], ORC_NODE_V, i + 1, j, wb);
        flux_y(gamma, wa, fa);
        flux_y(gamma, wm, fm);
        flux_y(gamma, wb, fb);
        for (int k = 0; k < 4; ++k) ghat[k] += tw[s] * (fa[k] + 4.0 * fm[k] + fb[k]) / 6.0;
      }
      for (int k = 0; k < 4; ++k) {
        fx[(size_t)k * N + id] = fhat[k];
        gy[(size_t)k * N + id] = ghat[k];
      }
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t id = (size_t)j * nx + i;
      size_t ip = (size_t)j * nx + wrap(i + 1, nx);
      size_t jp = (size_t)wrap(j + 1, ny) * nx + i;
      for (int k = 0; k < 4; ++k) {
        const double *F = fx + (size_t)k * N, *G = gy + (size_t)k * N;
        out[(size_t)k * N + id] =
            in[(size_t)k * N + id] - dt / h * (F[ip] - F[id]) - dt / h * (G[jp] - G[id]);
      }
    }
  for (size_t k = 0; k < 16 * N; ++k)
    if (!isfinite(out[k])) {
      flags |= ORC_FLAG_NONFINITE;
      break;
    }
  free(fx);
  free(gy);
  free(wc);
  free(ac);
  free(dd);
  free(half);
  return flags;
}

int orc_run(int nx, int ny, double h, double gamma, double dt, int variant, int n_steps,
            double *state) {
  size_t N = (size_t)nx * ny;
  double *tmp = (double *)malloc(sizeof(double) * 16 * N);
  int flags = 0;
  for (int n = 0; n < n_steps; ++n) {
    flags |= orc_step(nx, ny, h, gamma, dt, variant, state, tmp);
    memcpy(state, tmp, sizeof(double) * 16 * N);
  }
  free(tmp);
  return flags;
}

/* ------------------------------------------------------------------------ */
/* Global diagnostics in FP64.  out[ORC_NINV]:                               */
/*  0..3  h^2 sum of the cell averages (mass, x-, y-momentum, energy): the   */
/*        quantities the flux-difference update conserves (Sec. 3.1)          */
/*  4     entropy functional -int rho log(p / rho^gamma) dA (Sec. 6) by the  */
/*        tensor Simpson rule on each cell's nine primitive nodes            */
/*  5     the same functional from the cell averages (one point per cell)    */
/*  6     kinetic energy h^2 sum (m_x^2 + m_y^2) / (2 rho) of the averages    */
/*  7     max over V, E_v, E_h and centre nodes of sqrt(u^2+v^2) + c          */
/*  8,9   min rho, min p over the same nodes                                 */
/*  10    int (v_x - u_y) dA: Simpson along each cell edge (exact for the    */
/*        edge restrictions of the Q2 reconstruction), Sec. 6.4              */
/*  11    ORC_FLAG_* seen by the centre recovery                             */
/* ------------------------------------------------------------------------ */
static double entropy_density(double gamma, const double *w) {
  return -w[0] * log(w[3] / pow(w[0], gamma));
}

void orc_invariants(int nx, int ny, double h, double gamma, const double *st, double *out) {
  size_t N = (size_t)nx * ny;
  double *wc = (double *)malloc(sizeof(double) * 4 * N);
  int flags = orc_center_recovery(nx, ny, gamma, st, wc);
  double cons[4] = {0, 0, 0, 0}, ent = 0, enta = 0, ke = 0, smax = 0;
  double rmin = INFINITY, pmin = INFINITY, vort = 0;
  const double sw[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t id = (size_t)j * nx + i;
      double ub[4];
      for (int k = 0; k < 4; ++k) {
        ub[k] = st[(size_t)k * N + id];
        cons[k] += ub[k];
      }
      double wa[4];
      cons_to_prim(gamma, ub, wa);
      enta += entropy_density(gamma, wa);
      ke += 0.5 * (ub[1] * ub[1] + ub[2] * ub[2]) / ub[0];
      double f[3][3][4];
      cell_nodes(nx, ny, st, wc, i, j, f);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) ent += sw[a] * sw[b] * entropy_density(gamma, f[a][b]);
      /* nodes owned by this cell: V(i,j) = f[0][0], E_h(i,j) = f[1][0],
       * E_v(i,j) = f[0][1], centre f[1][1] */
      const double *own[4] = {f[0][0], f[1][0], f[0][1], f[1][1]};
      for (int k = 0; k < 4; ++k) {
        const double *w = own[k];
        double c = sqrt(gamma * w[3] / w[0]);
        double s = sqrt(w[1] * w[1] + w[2] * w[2]) + c;
        if (s > smax) smax = s;
        if (w[0] < rmin) rmin = w[0];
        if (w[3] < pmin) pmin = w[3];
      }
      /* int_C v_x = int_y [v(x_{i+1},y) - v(x_i,y)] dy ; int_C u_y likewise */
      double vr = 0, vl = 0, ut = 0, ubt = 0;
      for (int b = 0; b < 3; ++b) {
        vr += sw[b] * f[2][b][2];
        vl += sw[b] * f[0][b][2];
      }
      for (int a = 0; a < 3; ++a) {
        ut += sw[a] * f[a][2][1];
        ubt += sw[a] * f[a][0][1];
      }
      vort += h * (vr - vl) - h * (ut - ubt);
    }
  double h2 = h * h;
  for (int k = 0; k < 4; ++k) out[k] = h2 * cons[k];
  out[4] = h2 * ent;
  out[5] = h2 * enta;
  out[6] = h2 * ke;
  out[7] = smax;
  out[8] = rmin;
  out[9] = pmin;
  out[10] = vort;
  out[11] = (double)flags;
  free(wc);
}
