// af_fc.cuh -- foot-centred exact frozen acoustic point update (Appendix C),
// FP64 only: an analytical reference variant of the point update, not a hot
// path (the paper measures it at about 1000x the cost of the node-centred one).
//
// For a target point P and a duration tau the convective foot F comes from the
// same two Picard stages as the transported update; the acoustic state is
// frozen at F (W_* = R_h W(F), c_*, Z_* = rho_* c_*; Eq. fc-foot-freeze) and the
// disk of radius R = c_* tau is centred at F.  Under the compact footprint
// condition |F - P|_x + R < h/2, |F - P|_y + R < h/2 (Eq. fc-half-footprint)
// the disk is cut only by the grid lines through P: a vertex disk into the four
// cells around P, an edge disk into the two cells beside the edge.
//
// The exact solution of frozen linear acoustics (u_t + c grad pi = 0,
// pi_t + c div u = 0, pi = p / Z_*) at the centre of the disk, for continuous
// piecewise-Q2 data in monomials about F (units of h), is
//   pi(F) = sum_frag sum_ab r^q [ P_ab E_ab - a U_ab m_{a-1,b} - b V_ab m_{a,b-1} ] / 4pi
//   u(F)  = u_0(F) + sum_frag sum_ab { r^q [ -a P_ab m_{a-1,b} + a U_ab m_ab
//             + a V_ab m_{a-1,b+1} ] + a U_ab h_ab + a V_ab h_{a-1,b+1} } / 4pi
//   v(F)  = v_0(F) + (the same with the roles of the axes exchanged)
// with q = a + b, r = R/h, and for each fragment (scaled to the unit disk) its
// area moments m_ij = int xi^i eta^j Psi (Psi = 2 (1 - |w|^2)^{-1/2}, the
// projected-sphere weight), its radius derivative E_ab = r^-q d/dr (r^{q+1} m_ab)
// and its history h_ij = int_0^r s^{q-1} m_ij(s) ds (Eq. fc-moment-families).
//
// The fragments are assembled from three primitives by inclusion-exclusion
// (Eq. fc-role-rows): the full disk (closed form), the single cap {xi >= a}
// (closed form: a polynomial in a), the double cap {xi >= a, eta >= b}; caps on
// the other side of a line follow by reflection (moments times (-1)^i or
// (-1)^j) and complement.  The double cap is sliced into circles of projected
// radius p around F: on each circle the cap is one arc whose angular moments
// are closed forms, and the integral over p is taken by tanh-sinh quadrature
// (the integrands end in square-root singularities at both ends of the p-range).
#pragma once

#include "af_ref_kernels.cuh"

namespace af {
namespace fc {

constexpr int NM = 5;  // moment indices i + j <= 4
constexpr double PI = 3.14159265358979323846;

struct Moments {
  double m[NM][NM];  // area moments
  double e[3][3];    // radius derivative r^-q d/dr (r^{q+1} m_ab)
  double h[NM][NM];  // history int_0^r s^{q-1} m_ij(s) ds
};

__device__ __forceinline__ void clear(Moments& M) {
  for (int i = 0; i < NM; ++i)
    for (int j = 0; j < NM; ++j) M.m[i][j] = M.h[i][j] = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M.e[i][j] = 0.0;
}

__device__ __forceinline__ double ipow(double x, int n) {
  double r = 1.0;
  for (int k = 0; k < n; ++k) r *= x;
  return r;
}

// out += c * (reflected in), reflection signs (-1)^(i rx + j ry)
__device__ __forceinline__ void axpy(Moments& out, double c, const Moments& in, int rx, int ry) {
  for (int i = 0; i < NM; ++i)
    for (int j = 0; i + j < NM; ++j) {
      const double s = (((i * rx + j * ry) & 1) ? -c : c);
      out.m[i][j] += s * in.m[i][j];
      out.h[i][j] += s * in.h[i][j];
      if (i < 3 && j < 3) out.e[i][j] += s * in.e[i][j];
    }
}

__device__ __forceinline__ void transpose(Moments& M) {
  for (int i = 0; i < NM; ++i)
    for (int j = i + 1; j < NM; ++j) {
      double t = M.m[i][j];
      M.m[i][j] = M.m[j][i];
      M.m[j][i] = t;
      t = M.h[i][j];
      M.h[i][j] = M.h[j][i];
      M.h[j][i] = t;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j) {
      double t = M.e[i][j];
      M.e[i][j] = M.e[j][i];
      M.e[j][i] = t;
    }
}

// Full disk: the moments of the unit sphere, int w1^i w2^j dA = 4pi (1),
// 4pi/3 (w1^2), 4pi/5 (w1^4), 4pi/15 (w1^2 w2^2); zero for odd powers.
__device__ void full_disk(double r, Moments& M) {
  clear(M);
  M.m[0][0] = 4.0 * PI;
  M.m[2][0] = M.m[0][2] = 4.0 * PI / 3.0;
  M.m[4][0] = M.m[0][4] = 4.0 * PI / 5.0;
  M.m[2][2] = 4.0 * PI / 15.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M.e[i][j] = (i + j + 1) * M.m[i][j];
  for (int i = 0; i < NM; ++i)
    for (int j = 0; i + j < NM; ++j)
      if (i + j >= 1) M.h[i][j] = ipow(r, i + j) / (i + j) * M.m[i][j];
}

// Single cap {xi >= a}, 0 <= a: slicing at fixed xi, the chord carries
// int eta^j Psi d eta = 2 (1 - xi^2)^{j/2} J_j, J_0 = pi, J_2 = pi/2,
// J_4 = 3pi/8 (odd j: 0), so m_ij(a) = 2 J_j int_a^1 xi^i (1 - xi^2)^{j/2} d xi,
// a sum of terms c_k a^k.
__device__ void single_cap(double a, double r, Moments& M) {
  clear(M);
  if (a >= 1.0) return;
  const double d = a * r;  // offset of the line in units of h
  for (int i = 0; i < NM; ++i)
    for (int j = 0; i + j < NM; j += 2) {
      double c[4];
      int k[4], nt;
      const double ip1 = i + 1.0, ip3 = i + 3.0, ip5 = i + 5.0;
      if (j == 0) {
        c[0] = 2.0 * PI / ip1; k[0] = 0;
        c[1] = -2.0 * PI / ip1; k[1] = i + 1;
        nt = 2;
      } else if (j == 2) {
        c[0] = PI / ip1 - PI / ip3; k[0] = 0;
        c[1] = -PI / ip1; k[1] = i + 1;
        c[2] = PI / ip3; k[2] = i + 3;
        nt = 3;
      } else {  // j == 4: (1 - xi^2)^2 = 1 - 2 xi^2 + xi^4, 2 J_4 = 3pi/4
        const double w = 0.75 * PI;
        c[0] = w * (1.0 / ip1 - 2.0 / ip3 + 1.0 / ip5); k[0] = 0;
        c[1] = -w / ip1; k[1] = i + 1;
        c[2] = 2.0 * w / ip3; k[2] = i + 3;
        c[3] = -w / ip5; k[3] = i + 5;
        nt = 4;
      }
      double m = 0.0;
      for (int t = 0; t < nt; ++t) m += c[t] * ipow(a, k[t]);
      M.m[i][j] = m;
      const int q = i + j;
      if (q >= 1) {
        // h = sum_k c_k d^k int_d^r s^{q-1-k} ds (the cap is empty for s < d)
        double hv = 0.0;
        for (int t = 0; t < nt; ++t) {
          if (k[t] > 0 && d == 0.0) continue;
          const int ex = q - k[t];  // never 0 here
          const double dk = ipow(d, k[t]);
          const double rp = ex > 0 ? ipow(r, ex) : 1.0 / ipow(r, -ex);
          const double dp = ex > 0 ? ipow(d, ex) : 1.0 / ipow(d, -ex);
          hv += c[t] * dk * (rp - dp) / ex;
        }
        M.h[i][j] = hv;
      }
      if (i < 3 && j < 3) {
        // r d/dr of m(a = d/r) is -a dm/da = a * 2 J_j a^i (1 - a^2)^{j/2}
        const double Jj = j == 0 ? PI : 0.5 * PI;
        M.e[i][j] = (q + 1) * m + 2.0 * Jj * ipow(a, i + 1) * ipow(1.0 - a * a, j / 2);
      }
    }
}

// T[i][j] = int_0^phi cos^i sin^j, i + j <= 4, from the reduction formulas.
__device__ void arc_table(double phi, double T[NM][NM]) {
  double s, c;
  sincos(phi, &s, &c);
  T[0][0] = phi;
  T[1][0] = s;
  T[0][1] = 1.0 - c;
  T[1][1] = 0.5 * s * s;
  // reduce the sine power while it is at least 2, else the cosine power (then
  // i >= 2, since n >= 2 and (1, 1) is a base case)
  for (int n = 2; n < NM; ++n)
    for (int i = 0; i <= n; ++i) {
      const int j = n - i;
      if (i == 1 && j == 1) continue;
      if (j >= 2)
        T[i][j] = (-ipow(s, j - 1) * ipow(c, i + 1) + (j - 1) * T[i][j - 2]) / n;
      else
        T[i][j] = (ipow(c, i - 1) * ipow(s, j + 1) + (i - 1) * T[i - 2][j]) / n;
    }
}

// int_0^{asin x} sin^j, j <= 2
__device__ __forceinline__ double sin_int(int j, double x) {
  const double c = sqrt(fmax(1.0 - x * x, 0.0)), ph = asin(x);
  return j == 0 ? ph : (j == 1 ? 1.0 - c : 0.5 * (ph - x * c));
}

// Double cap {xi >= a, eta >= b}, a, b >= 0.  On the circle of projected radius
// p the cap is the arc [asin(b/p), acos(a/p)]; with A_ij(p) its angular moment,
//   m_ij = 2 int p^{q+1} A_ij(p) / sqrt(1 - p^2) dp,
//   h_ij = 2 r^q int p^{q-1} sqrt(1 - p^2) A_ij(p) dp,   p in [sqrt(a^2+b^2), 1],
// and E from the line integrals along the two cut lines.
__device__ void double_cap(double a, double b, double r, Moments& M) {
  clear(M);
  const double pb2 = a * a + b * b;
  if (pb2 >= 1.0) return;
  const double pb = sqrt(pb2), L = 1.0 - pb;
  // tanh-sinh rule on [0, 1]: nodes x = 1/(1 + e^{-2u}), u = (pi/2) sinh(k/16)
  for (int kk = -64; kk <= 64; ++kk) {
    const double t = kk * (1.0 / 16.0);
    const double u = 0.5 * PI * sinh(t);
    const double cu = cosh(u);
    const double w = 0.5 * (1.0 / 16.0) * 0.5 * PI * cosh(t) / (cu * cu);
    if (!(w > 1e-300)) continue;
    const double x = 1.0 / (1.0 + exp(-2.0 * u)), omx = 1.0 / (1.0 + exp(2.0 * u));
    const double p = pb + L * x, omp = L * omx;
    const double sq = sqrt(omp * (1.0 + p));
    if (!(p > 0.0) || !(sq > 0.0)) continue;
    const double ph1 = asin(fmin(b / p, 1.0)), ph2 = acos(fmin(a / p, 1.0));
    if (!(ph2 > ph1)) continue;
    double T1[NM][NM], T2[NM][NM];
    arc_table(ph1, T1);
    arc_table(ph2, T2);
    const double wl = L * w;
    for (int i = 0; i < NM; ++i)
      for (int j = 0; i + j < NM; ++j) {
        const int q = i + j;
        const double A = T2[i][j] - T1[i][j];
        M.m[i][j] += wl * 2.0 * ipow(p, q + 1) * A / sq;
        if (q >= 1) M.h[i][j] += wl * 2.0 * ipow(r, q) * ipow(p, q - 1) * sq * A;
      }
  }
  // r d/dr m(a = dx/r, b = dy/r) = -a dm/da - b dm/db; the derivatives are
  // minus the line integrals of xi^i eta^j Psi along xi = a and eta = b
  const double sa = sqrt(1.0 - a * a), sb = sqrt(1.0 - b * b);
  const double half[3] = {0.5 * PI, 1.0, 0.25 * PI};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double la = ipow(a, i) * 2.0 * ipow(sa, j) * (half[j] - sin_int(j, fmin(b / sa, 1.0)));
      const double lb = ipow(b, j) * 2.0 * ipow(sb, i) * (half[i] - sin_int(i, fmin(a / sb, 1.0)));
      M.e[i][j] = (i + j + 1) * M.m[i][j] + a * la + b * lb;
    }
}

// Region {xi >= lam} for any lam (cap, or complement of the reflected cap).
__device__ void region_x(double lam, double r, const Moments& F, Moments& out) {
  Moments c;
  if (lam >= 0.0) {
    single_cap(lam, r, out);
    return;
  }
  single_cap(-lam, r, c);
  clear(out);
  axpy(out, 1.0, F, 0, 0);
  axpy(out, -1.0, c, 1, 0);
}

__device__ void region_y(double mu, double r, const Moments& F, Moments& out) {
  region_x(mu, r, F, out);  // the full disk is symmetric
  transpose(out);
}

// Region {xi >= lam, eta >= mu} for any signs.
__device__ void region_xy(double lam, double mu, double r, const Moments& F, const Moments& X,
                          const Moments& Y, Moments& out) {
  Moments c;
  double_cap(fabs(lam), fabs(mu), r, c);
  clear(out);
  if (lam >= 0.0 && mu >= 0.0) {
    axpy(out, 1.0, c, 0, 0);
  } else if (lam < 0.0 && mu >= 0.0) {  // {eta >= mu} minus {xi < lam, eta >= mu}
    axpy(out, 1.0, Y, 0, 0);
    axpy(out, -1.0, c, 1, 0);
  } else if (lam >= 0.0 && mu < 0.0) {
    axpy(out, 1.0, X, 0, 0);
    axpy(out, -1.0, c, 0, 1);
  } else {  // complement of {xi < lam} u {eta < mu}
    Moments cx, cy;
    single_cap(-lam, r, cx);
    single_cap(-mu, r, cy);
    transpose(cy);
    axpy(out, 1.0, F, 0, 0);
    axpy(out, -1.0, cx, 1, 0);
    axpy(out, -1.0, cy, 0, 1);
    axpy(out, 1.0, c, 1, 1);
  }
}

// Coefficients (1, X, X^2) of the Q2 Lagrange basis l_0, l_1, l_2 at local
// coordinate s = sF + 2X (X the offset from F in units of h).
__device__ __forceinline__ void basis_about(double sF, double B[3][3]) {
  B[0][0] = 0.5 * sF * (sF - 1.0); B[0][1] = 2.0 * sF - 1.0; B[0][2] = 2.0;
  B[1][0] = 1.0 - sF * sF;         B[1][1] = -4.0 * sF;      B[1][2] = -4.0;
  B[2][0] = 0.5 * sF * (sF + 1.0); B[2][1] = 2.0 * sF + 1.0; B[2][2] = 2.0;
}

// Adds one fragment's contribution to (pi, u, v) * 4pi; P, U, V are its
// (pi, u, v) deviations in monomials about F.
__device__ void contract(const Moments& M, const double P[3][3], const double U[3][3],
                         const double V[3][3], double r, double acc[3]) {
  auto mm = [&](int i, int j) { return (i < 0 || j < 0) ? 0.0 : M.m[i][j]; };
  auto hh = [&](int i, int j) { return (i < 0 || j < 0) ? 0.0 : M.h[i][j]; };
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const double rq = ipow(r, a + b);
      acc[0] += rq * (P[a][b] * M.e[a][b] - a * U[a][b] * mm(a - 1, b) - b * V[a][b] * mm(a, b - 1));
      acc[1] += rq * (-a * P[a][b] * mm(a - 1, b) + a * U[a][b] * mm(a, b) +
                      a * V[a][b] * mm(a - 1, b + 1)) +
                a * U[a][b] * hh(a, b) + a * V[a][b] * hh(a - 1, b + 1);
      acc[2] += rq * (-b * P[a][b] * mm(a, b - 1) + b * U[a][b] * mm(a + 1, b - 1) +
                      b * V[a][b] * mm(a, b)) +
                b * U[a][b] * hh(a + 1, b - 1) + b * V[a][b] * hh(a, b);
    }
}

}  // namespace fc

// Foot-centred point update of family FAM (0 V, 1 E_v, 2 E_h), FP64, one thread
// per point, both durations; writes the half-step and new point planes.
template <int FAM>
__global__ void k_points_fc(StepArgs<double> a) {
  using namespace fc;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  LatticeG<double> L = lattice_of(a);
  const int I = 2 * i + (FAM == 2 ? 1 : 0);
  const int J = 2 * j + (FAM == 1 ? 1 : 0);
  const Prim<double> wp = L.at(I, J);
  const size_t id = (size_t)j * a.nx + i;
  const double hinv = 1.0 / a.h;
  // adjacent cells (lower-left lattice corner) and their side of the lines x = x_P, y = y_P
  constexpr int NF = FAM == 0 ? 4 : 2;
  int cI[NF], cJ[NF], sx[NF], sy[NF];
  if (FAM == 0) {
    const int dI[4] = {0, -2, -2, 0}, dJ[4] = {0, 0, -2, -2};
    const int ex[4] = {1, -1, -1, 1}, ey[4] = {1, 1, -1, -1};
    for (int k = 0; k < 4; ++k) {
      cI[k] = I + dI[k]; cJ[k] = J + dJ[k]; sx[k] = ex[k]; sy[k] = ey[k];
    }
  } else if (FAM == 1) {  // E_v(i,j): right C(i,j), left C(i-1,j)
    cI[0] = I; cJ[0] = J - 1; sx[0] = 1; sy[0] = 0;
    cI[1] = I - 2; cJ[1] = J - 1; sx[1] = -1; sy[1] = 0;
  } else {  // E_h(i,j): upper C(i,j), lower C(i,j-1)
    cI[0] = I - 1; cJ[0] = J; sx[0] = 0; sy[0] = 1;
    cI[1] = I - 1; cJ[1] = J - 2; sx[1] = 0; sy[1] = -1;
  }
  unsigned bad = 0;
  for (int s = 0; s < 2; ++s) {
    const double tau = s == 0 ? 0.5 * a.dt : a.dt;
    const double th = tau * hinv;
    // two-Picard convective foot (Eq. adv-footpoint), then the frozen state at F
    const double d1x = -th * wp.u, d1y = -th * wp.v;
    const Prim<double> w1 = eval_w(L, locate<double>(I, J, d1x, d1y));
    const double fx = -th * w1.u, fy = -th * w1.v;  // F - P, units of h
    const Prim<double> ws = eval_w(L, locate<double>(I, J, fx, fy));
    if (!(ws.r > 0.0 && ws.p > 0.0)) bad |= FLAG_NONPHYSICAL;
    const double cs = sqrt(a.gas.gamma * ws.p / ws.r), Z = ws.r * cs;
    const double r = cs * th;
    if (!(fabs(fx) + r < 0.5 && fabs(fy) + r < 0.5)) bad |= FLAG_CFL | FLAG_REACH;
    const double rr = fmax(r, 1e-300);
    const double lam = -fx / rr, mu = -fy / rr;  // the lines through P, scaled
    Moments Fm, X, Y, XY;
    full_disk(rr, Fm);
    if (FAM != 2) region_x(lam, rr, Fm, X);
    if (FAM != 1) region_y(mu, rr, Fm, Y);
    if (FAM == 0) region_xy(lam, mu, rr, Fm, X, Y, XY);
    double acc[3] = {0.0, 0.0, 0.0}, u0 = 0.0, v0 = 0.0;
    for (int k = 0; k < NF; ++k) {
      // the fragment: inclusion-exclusion of the primitives (Eq. fc-role-rows)
      Moments G;
      clear(G);
      if (FAM == 0) {
        const bool px = sx[k] > 0, py = sy[k] > 0;
        if (px && py) { axpy(G, 1.0, XY, 0, 0); }
        else if (!px && py) { axpy(G, 1.0, Y, 0, 0); axpy(G, -1.0, XY, 0, 0); }
        else if (px) { axpy(G, 1.0, X, 0, 0); axpy(G, -1.0, XY, 0, 0); }
        else {
          axpy(G, 1.0, Fm, 0, 0); axpy(G, -1.0, X, 0, 0); axpy(G, -1.0, Y, 0, 0);
          axpy(G, 1.0, XY, 0, 0);
        }
      } else {
        const Moments& C = FAM == 1 ? X : Y;
        const int side = FAM == 1 ? sx[k] : sy[k];
        if (side > 0) { axpy(G, 1.0, C, 0, 0); }
        else { axpy(G, 1.0, Fm, 0, 0); axpy(G, -1.0, C, 0, 0); }
      }
      // the cell's Q2 data as deviations from W_*, in monomials about F
      double Bx[3][3], By[3][3];
      basis_about((double)(I - cI[k] - 1) + 2.0 * fx, Bx);
      basis_about((double)(J - cJ[k] - 1) + 2.0 * fy, By);
      double P[3][3] = {}, U[3][3] = {}, V[3][3] = {};
      for (int ix = 0; ix < 3; ++ix)
        for (int iy = 0; iy < 3; ++iy) {
          const Prim<double> w = L.at(cI[k] + ix, cJ[k] + iy);
          const double dp = (w.p - ws.p) / Z, du = w.u - ws.u, dv = w.v - ws.v;
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) {
              const double bb = Bx[ix][p] * By[iy][q];
              P[p][q] += dp * bb;
              U[p][q] += du * bb;
              V[p][q] += dv * bb;
            }
        }
      // the cell holding F gives the data value at F
      const bool holds = (FAM == 2 || sx[k] * (-fx) <= 0.0) && (FAM == 1 || sy[k] * (-fy) <= 0.0);
      if (holds) {
        u0 = U[0][0];
        v0 = V[0][0];
      }
      contract(G, P, U, V, rr, acc);
    }
    Prim<double> nw;
    const double k4 = 1.0 / (4.0 * PI);
    nw.p = ws.p + Z * (acc[0] * k4);
    nw.u = ws.u + (u0 + acc[1] * k4);
    nw.v = ws.v + (v0 + acc[2] * k4);
    nw.r = ws.r + (nw.p - ws.p) / (cs * cs);
    if (!(isfinite(nw.r) && isfinite(nw.u) && isfinite(nw.v) && isfinite(nw.p)))
      bad |= FLAG_NONFINITE;
    double* const* dst = s == 0 ? a.half[FAM] : a.out.pt[FAM];
    dst[0][id] = nw.r;
    dst[1][id] = nw.u;
    dst[2][id] = nw.v;
    dst[3][id] = nw.p;
  }
  raise_flag(a.flags, bad);
}

}  // namespace af
