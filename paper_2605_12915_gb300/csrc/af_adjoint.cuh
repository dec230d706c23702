// af_adjoint.cuh -- hand-written discrete adjoint of one step (Sec. 6.1):
// lambda^n = (d state^{n+1} / d state^n)^T lambda^{n+1}, linearised about the
// state at t^n.  The forward intermediates are recomputed by the unfused step
// kernels (af_ref_kernels.cuh); the reverse sweep then runs, one thread per
// cell, through
//   k_adj_flux      average update and space-time Simpson fluxes (gather)
//   k_adj_points    transported / additive point update, Q2 evaluation at the
//                   foot, the two Picard stages (scatter with atomics)
//   k_adj_acoustic  Horner in r, node freezing (c, Z, r) and the transposed
//                   acoustic stencils (scatter)
//   k_adj_center    Simpson inversion (scatter)
// Adjoints are with respect to the stored variables; the storage offsets of
// the FP32 modes are constant shifts and do not change them.
#pragma once

#include "af_common.cuh"
#include "af_ref_kernels.cuh"

namespace af {

__device__ __forceinline__ void atomic_add(float* p, float v) {
  if (v != 0.f) atomicAdd(p, v);
}
__device__ __forceinline__ void atomic_add(double* p, double v) {
  if (v != 0.0) atomicAdd(p, v);
}

template <typename T>
struct AdjArgs {
  StepArgs<T> f;       // forward arguments: in = state^n, intermediates recomputed
  T* lin[16];          // lambda^{n+1}: averages 0-3, V 4-7, E_v 8-11, E_h 12-15
  T* lout[16];         // lambda^n (same layout)
  T* lwc[4];           // adjoint of the recovered centres
  T* linc[2][4][3];    // adjoint of the increments [tau][family][du, dv, dp]
  T* lhalf[3][4];      // adjoint of the half-step point values
  T* lfull[3][4];      // adjoint of the full-step point values
};

// adjoint of a lattice of (rho, u, v, p): families 0-2 are points, 3 the centres
template <typename T>
struct LatticeAdj {
  T* f[4][4];
  int nx, ny;
  __device__ __forceinline__ void add(int I, int J, T r, T u, T v, T p) const {
    const int fam = lattice_family(I, J);
    const size_t id = (size_t)wrapi(J >> 1, ny) * nx + wrapi(I >> 1, nx);
    atomic_add(f[fam][0] + id, r);
    atomic_add(f[fam][1] + id, u);
    atomic_add(f[fam][2] + id, v);
    atomic_add(f[fam][3] + id, p);
  }
};

template <typename T>
__device__ __forceinline__ LatticeAdj<T> lattice_adj_of(const AdjArgs<T>& a) {
  LatticeAdj<T> L;
  for (int f = 0; f < 3; ++f)
    for (int k = 0; k < 4; ++k) L.f[f][k] = a.lout[4 + 4 * f + k];
  for (int k = 0; k < 4; ++k) L.f[3][k] = a.lwc[k];
  L.nx = a.f.nx;
  L.ny = a.f.ny;
  return L;
}

// Transposed Euler flux Jacobians: out += J_F(w)^T l  (stored primitives)
template <typename T>
__device__ __forceinline__ void flux_x_adj(const Prim<T>& w, const Gas<T>& g, const T l[4],
                                           T s, T o[4]) {
  const T rho = g.rho_ref + w.r, p = g.p_ref + w.p;
  const T q2 = w.u * w.u + w.v * w.v;
  const T hh = p * g.g_gm1 + T(0.5) * rho * q2;
  o[0] += s * (w.u * l[0] + w.u * w.u * l[1] + w.u * w.v * l[2] + T(0.5) * w.u * q2 * l[3]);
  o[1] += s * (rho * l[0] + T(2) * rho * w.u * l[1] + rho * w.v * l[2] +
               (hh + rho * w.u * w.u) * l[3]);
  o[2] += s * (rho * w.u * l[2] + rho * w.u * w.v * l[3]);
  o[3] += s * (l[1] + g.g_gm1 * w.u * l[3]);
}

template <typename T>
__device__ __forceinline__ void flux_y_adj(const Prim<T>& w, const Gas<T>& g, const T l[4],
                                           T s, T o[4]) {
  const T rho = g.rho_ref + w.r, p = g.p_ref + w.p;
  const T q2 = w.u * w.u + w.v * w.v;
  const T hh = p * g.g_gm1 + T(0.5) * rho * q2;
  o[0] += s * (w.v * l[0] + w.u * w.v * l[1] + w.v * w.v * l[2] + T(0.5) * w.v * q2 * l[3]);
  o[1] += s * (rho * w.v * l[1] + rho * w.u * w.v * l[3]);
  o[2] += s * (rho * l[0] + rho * w.u * l[1] + T(2) * rho * w.v * l[2] +
               (hh + rho * w.v * w.v) * l[3]);
  o[3] += s * (l[2] + g.g_gm1 * w.v * l[3]);
}

// ---------------------------------------------------------------------------
// Average update and fluxes (Eq. af-average-update), gathered per cell: the
// adjoints of the three point families of cell (i,j) at sigma = 0, 1/2, 1.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_adj_flux(AdjArgs<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = a.f.nx, ny = a.f.ny;
  if (i >= nx || j >= ny) return;
  const int im = wrapi(i - 1, nx), jm = wrapi(j - 1, ny);
  const size_t id = (size_t)j * nx + i, idl = (size_t)j * nx + im, idb = (size_t)jm * nx + i,
               idlb = (size_t)jm * nx + im;
  T lfx[4], lfxb[4], lgy[4], lgyl[4];
  for (int k = 0; k < 4; ++k) {
    const T c = a.lin[k][id], l = a.lin[k][idl], b = a.lin[k][idb], lb = a.lin[k][idlb];
    lfx[k] = c - l;    // vertical edge x_i of cell (i,j)
    lfxb[k] = b - lb;  // vertical edge x_i of cell (i,j-1)
    lgy[k] = c - b;    // horizontal edge y_j of cell (i,j)
    lgyl[k] = l - lb;  // horizontal edge y_j of cell (i-1,j)
    a.lout[k][id] = c;
  }
  const T cst = a.f.dt / (T(36) * a.f.h);
  const T wt[3] = {T(1), T(4), T(1)};
  T* const* lev[3][3] = {{a.f.in.pt[0], a.f.in.pt[1], a.f.in.pt[2]},
                         {a.f.half[0], a.f.half[1], a.f.half[2]},
                         {a.f.out.pt[0], a.f.out.pt[1], a.f.out.pt[2]}};
  T lvx[4], lvy[4];
  for (int k = 0; k < 4; ++k) {
    lvx[k] = lfx[k] + lfxb[k];
    lvy[k] = lgy[k] + lgyl[k];
  }
  for (int s = 0; s < 3; ++s) {
    const T sc = cst * wt[s];
    T oV[4] = {T(0), T(0), T(0), T(0)}, oEv[4] = {T(0), T(0), T(0), T(0)},
      oEh[4] = {T(0), T(0), T(0), T(0)};
    flux_x_adj(load_pt<T>(lev[s][0], id), a.f.gas, lvx, sc, oV);
    flux_y_adj(load_pt<T>(lev[s][0], id), a.f.gas, lvy, sc, oV);
    flux_x_adj(load_pt<T>(lev[s][1], id), a.f.gas, lfx, T(4) * sc, oEv);
    flux_y_adj(load_pt<T>(lev[s][2], id), a.f.gas, lgy, T(4) * sc, oEh);
    const T* oo[3] = {oV, oEv, oEh};
    for (int f = 0; f < 3; ++f)
      for (int k = 0; k < 4; ++k) {
        if (s == 0) a.lout[4 + 4 * f + k][id] = oo[f][k];
        else if (s == 1) a.lhalf[f][k][id] = oo[f][k];
        else a.lfull[f][k][id] = oo[f][k] + a.lin[4 + 4 * f + k][id];
      }
  }
}

// derivative of the Lagrange basis l_-, l_0, l_+ with respect to s
template <typename T>
__device__ __forceinline__ void lagrange3_d(T s, T d[3]) {
  d[0] = s - T(0.5);
  d[1] = T(-2) * s;
  d[2] = s + T(0.5);
}

template <typename T>
struct IncAdj {
  T* f[4][3];
  int nx, ny;
  __device__ __forceinline__ void add(int I, int J, T du, T dv, T dp) const {
    const int fam = lattice_family(I, J);
    const size_t id = (size_t)wrapi(J >> 1, ny) * nx + wrapi(I >> 1, nx);
    atomic_add(f[fam][0] + id, du);
    atomic_add(f[fam][1] + id, dv);
    atomic_add(f[fam][2] + id, dp);
  }
};

// ---------------------------------------------------------------------------
// Point update (Sec. 6.1 steps 3-4; Eq. barsukow-additive), reversed.
// ---------------------------------------------------------------------------
template <int FAM, typename T>
__global__ void k_adj_points(AdjArgs<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const StepArgs<T>& f = a.f;
  if (i >= f.nx || j >= f.ny) return;
  const LatticeG<T> L = lattice_of(f);
  const LatticeAdj<T> LA = lattice_adj_of(a);
  const int I = 2 * i + (FAM == 2 ? 1 : 0);
  const int J = 2 * j + (FAM == 1 ? 1 : 0);
  const Prim<T> wp = L.at(I, J);
  const size_t id = (size_t)j * f.nx + i;
  const T hinv = T(1) / f.h;
  const Gas<T>& g = f.gas;
  T luP = T(0), lvP = T(0), lrP = T(0), lpP = T(0);
  for (int s = 0; s < 2; ++s) {
    const T th = (s == 0 ? T(0.5) * f.dt : f.dt) * hinv;
    T* const* lsrc = s == 0 ? a.lhalf[FAM] : a.lfull[FAM];
    const T ly[4] = {lsrc[0][id], lsrc[1][id], lsrc[2][id], lsrc[3][id]};
    if (ly[0] == T(0) && ly[1] == T(0) && ly[2] == T(0) && ly[3] == T(0)) continue;
    IncrG<T> D;
    IncAdj<T> DA;
    for (int q = 0; q < 4; ++q)
      for (int k = 0; k < 3; ++k) {
        D.f[q][k] = f.inc[s][q][k];
        DA.f[q][k] = a.linc[s][q][k];
      }
    D.nx = DA.nx = f.nx;
    D.ny = DA.ny = f.ny;
    // forward recomputation of the foot (Eq. adv-footpoint)
    const T d1x = -th * wp.u, d1y = -th * wp.v;
    const FootCell<T> c1 = locate<T>(I, J, d1x, d1y);
    const Prim<T> w1 = eval_w(L, c1);
    const T dfx = -th * w1.u, dfy = -th * w1.v;
    const FootCell<T> fc = locate<T>(I, J, dfx, dfy);
    const Prim<T> wf = eval_w(L, fc);
    T lwf[4], ld[3];  // adjoints of W_f and of the interpolated increments
    if (f.variant == 0) {
      T d[3];
      eval_d(D, fc, d);
      const T rf = g.rho_ref + wf.r, pf = g.p_ref + wf.p;
      const T gp = g.gamma * pf;
      lwf[0] = ly[0] * (T(1) + d[2] / gp);
      lwf[1] = ly[1];
      lwf[2] = ly[2];
      lwf[3] = ly[3] - ly[0] * d[2] * rf / (gp * pf);
      ld[0] = ly[1];
      ld[1] = ly[2];
      ld[2] = ly[3] + ly[0] * rf / gp;
    } else {
      T d[3];
      D.at(I, J, d);
      const T rp = g.rho_ref + wp.r, pp = g.p_ref + wp.p;
      const T gp = g.gamma * pp;
      lwf[0] = ly[0];
      lwf[1] = ly[1];
      lwf[2] = ly[2];
      lwf[3] = ly[3];
      // nw.r = wf.r + dp rho_P / (gamma p_P), with the increments at P itself
      DA.add(I, J, ly[1], ly[2], ly[3] + ly[0] * rp / gp);
      lrP += ly[0] * d[2] / gp;
      lpP += -ly[0] * d[2] * rp / (gp * pp);
      ld[0] = ld[1] = ld[2] = T(0);
    }
    // scatter through the Q2 evaluation at the foot and collect the adjoint of
    // the foot's local coordinates
    T lx[3], lyb[3], dx3[3], dy3[3];
    lagrange3(fc.xi, lx);
    lagrange3(fc.eta, lyb);
    lagrange3_d(fc.xi, dx3);
    lagrange3_d(fc.eta, dy3);
    T lxi = T(0), leta = T(0);
    for (int b = 0; b < 3; ++b)
      for (int q = 0; q < 3; ++q) {
        const int In = 2 * fc.ci + q, Jn = 2 * fc.cj + b;
        const T wgt = lx[q] * lyb[b];
        LA.add(In, Jn, wgt * lwf[0], wgt * lwf[1], wgt * lwf[2], wgt * lwf[3]);
        const Prim<T> wn = L.at(In, Jn);
        T dot = wn.r * lwf[0] + wn.u * lwf[1] + wn.v * lwf[2] + wn.p * lwf[3];
        if (f.variant == 0) {
          DA.add(In, Jn, wgt * ld[0], wgt * ld[1], wgt * ld[2]);
          T dn[3];
          D.at(In, Jn, dn);
          dot += dn[0] * ld[0] + dn[1] * ld[1] + dn[2] * ld[2];
        }
        lxi += dx3[q] * lyb[b] * dot;
        leta += lx[q] * dy3[b] * dot;
      }
    // xi = 2 (foot - cell) - 1; the foot moved by df = -th (u1, v1)
    const T ldfx = T(2) * lxi, ldfy = T(2) * leta;
    const T lu1 = -th * ldfx, lv1 = -th * ldfy;
    // first Picard stage: (u1, v1) = R_h(u, v) at P + d1
    lagrange3(c1.xi, lx);
    lagrange3(c1.eta, lyb);
    lagrange3_d(c1.xi, dx3);
    lagrange3_d(c1.eta, dy3);
    lxi = T(0);
    leta = T(0);
    for (int b = 0; b < 3; ++b)
      for (int q = 0; q < 3; ++q) {
        const int In = 2 * c1.ci + q, Jn = 2 * c1.cj + b;
        const T wgt = lx[q] * lyb[b];
        LA.add(In, Jn, T(0), wgt * lu1, wgt * lv1, T(0));
        const Prim<T> wn = L.at(In, Jn);
        const T dot = wn.u * lu1 + wn.v * lv1;
        lxi += dx3[q] * lyb[b] * dot;
        leta += lx[q] * dy3[b] * dot;
      }
    const T ld1x = T(2) * lxi, ld1y = T(2) * leta;
    luP += -th * ld1x;
    lvP += -th * ld1y;
  }
  LA.add(I, J, lrP, luP, lvP, lpP);
}

// ---------------------------------------------------------------------------
// Acoustic increments (Sec. 6.1 step 1), reversed: Horner in r_s = c tau_s / h,
// freezing c = sqrt(gamma p / rho), Z = rho c, and the transposed stencils.
// ---------------------------------------------------------------------------
template <typename T>
struct ScatterLattice {
  const LatticeAdj<T>* LA;
  int I, J;
  __device__ __forceinline__ void operator()(int dx, int dy, T lp, T lu, T lv) const {
    LA->add(I + dx, J + dy, T(0), lu, lv, lp);
  }
};

template <int FAM, typename T, typename Scatter>
__device__ __forceinline__ void sac_family_adj(const Scatter& S, const T lGp[3][4],
                                               const T lGuv[3][4], T& lpK, T& luK, T& lvK) {
  if (FAM == 0) af_sac_V_adj<T>(S, lGp, lGuv, lpK, luK, lvK);
  if (FAM == 1) af_sac_EV_adj<T>(S, lGp, lGuv, lpK, luK, lvK);
  if (FAM == 2) af_sac_EH_adj<T>(S, lGp, lGuv, lpK, luK, lvK);
  if (FAM == 3) af_sac_C_adj<T>(S, lGp, lGuv, lpK, luK, lvK);
}

template <int FAM, typename T>
__global__ void k_adj_acoustic(AdjArgs<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const StepArgs<T>& f = a.f;
  if (i >= f.nx || j >= f.ny) return;
  const size_t id = (size_t)j * f.nx + i;
  T ld[2][3];
  bool any = false;
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      ld[s][k] = a.linc[s][FAM][k][id];
      any = any || ld[s][k] != T(0);
    }
  if (!any) return;
  const LatticeG<T> L = lattice_of(f);
  const LatticeAdj<T> LA = lattice_adj_of(a);
  const int I = 2 * i + ((FAM == 2 || FAM == 3) ? 1 : 0);
  const int J = 2 * j + ((FAM == 1 || FAM == 3) ? 1 : 0);
  const Prim<T> wk = L.at(I, J);
  const T rk = f.gas.rho_ref + wk.r, pk = f.gas.p_ref + wk.p;
  const T c = sqrt(f.gas.gamma * pk / rk);
  const T Z = rk * c, Zinv = T(1) / Z;
  const T dth = f.dt / f.h;
  const T r1 = c * dth;
  T Gp[3][4], Guv[3][4];
  LoadPUV<T> ldr = {&L, I, J};
  sac_family<FAM, T>(ldr, wk.p, wk.u, wk.v, Gp, Guv);
  // polynomial coefficients c_o[q] (q = 1..4 stored at 0..3), as in increments_at
  T co[3][4];
  for (int q = 0; q < 4; ++q) {
    co[2][q] = fma(Z, Guv[0][q], Gp[0][q]);   // dp
    co[0][q] = fma(Zinv, Gp[1][q], Guv[1][q]);  // du
    co[1][q] = fma(Zinv, Gp[2][q], Guv[2][q]);  // dv
  }
  T lco[3][4] = {}, lr1 = T(0);
  for (int s = 0; s < 2; ++s) {
    const T rs = s == 0 ? T(0.5) * r1 : r1;
    const T sc = s == 0 ? T(0.5) : T(1);
    T pw[5];
    pw[0] = T(1);
    for (int q = 1; q <= 4; ++q) pw[q] = pw[q - 1] * rs;
    for (int o = 0; o < 3; ++o) {
      T dr = T(0);
      for (int q = 1; q <= 4; ++q) {
        lco[o][q - 1] += pw[q] * ld[s][o];
        dr += T(q) * pw[q - 1] * co[o][q - 1];
      }
      lr1 += sc * dr * ld[s][o];
    }
  }
  T lGp[3][4], lGuv[3][4], lZ = T(0), lZinv = T(0);
  for (int q = 0; q < 4; ++q) {
    lGp[0][q] = lco[2][q];
    lGuv[0][q] = Z * lco[2][q];
    lZ += Guv[0][q] * lco[2][q];
    lGp[1][q] = Zinv * lco[0][q];
    lGuv[1][q] = lco[0][q];
    lZinv += Gp[1][q] * lco[0][q];
    lGp[2][q] = Zinv * lco[1][q];
    lGuv[2][q] = lco[1][q];
    lZinv += Gp[2][q] * lco[1][q];
  }
  lZ -= lZinv * Zinv * Zinv;
  const T lc = dth * lr1 + rk * lZ;
  T lrho = c * lZ - lc * c / (T(2) * rk);
  T lp = lc * c / (T(2) * pk);
  T lpK = T(0), luK = T(0), lvK = T(0);
  ScatterLattice<T> S = {&LA, I, J};
  sac_family_adj<FAM, T>(S, lGp, lGuv, lpK, luK, lvK);
  LA.add(I, J, lrho, luK, lvK, lp + lpK);
}

// ---------------------------------------------------------------------------
// Centre recovery (Eq. center-node), reversed.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void dcons_dprim_T(const Prim<T>& w, const Gas<T>& g, const T l[4],
                                              T s, T o[4]) {
  // o += s (dU/dW)^T l, U = (rho~, rho u, rho v, E~) of the stored primitive
  const T rho = g.rho_ref + w.r;
  o[0] += s * (l[0] + w.u * l[1] + w.v * l[2] + T(0.5) * (w.u * w.u + w.v * w.v) * l[3]);
  o[1] += s * (rho * l[1] + rho * w.u * l[3]);
  o[2] += s * (rho * l[2] + rho * w.v * l[3]);
  o[3] += s * (g.gm1inv * l[3]);
}

template <typename T, bool COMP>
__global__ void k_adj_center(AdjArgs<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const StepArgs<T>& f = a.f;
  if (i >= f.nx || j >= f.ny) return;
  const size_t id = (size_t)j * f.nx + i;
  const T lw[4] = {a.lwc[0][id], a.lwc[1][id], a.lwc[2][id], a.lwc[3][id]};
  if (lw[0] == T(0) && lw[1] == T(0) && lw[2] == T(0) && lw[3] == T(0)) return;
  const Gas<T>& g = f.gas;
  // the recovered centre (rho~, u, v, p~) is W(U_c); lambda_U = (dW/dU)^T lambda_W
  const T rho = g.rho_ref + f.wc[0][id], u = f.wc[1][id], v = f.wc[2][id];
  const T ri = T(1) / rho;
  T lU[4];
  lU[0] = lw[0] - u * ri * lw[1] - v * ri * lw[2] + g.gm1 * T(0.5) * (u * u + v * v) * lw[3];
  lU[1] = ri * lw[1] - g.gm1 * u * lw[3];
  lU[2] = ri * lw[2] - g.gm1 * v * lw[3];
  lU[3] = g.gm1 * lw[3];
  // U_c = 9/4 Ubar - 1/16 sum_corners U(W) - 1/4 sum_edges U(W)
  for (int k = 0; k < 4; ++k) atomic_add(a.lout[k] + id, T(2.25) * lU[k]);
  const LatticeAdj<T> LA = lattice_adj_of(a);
  const LatticeG<T> L = lattice_of(f);
  const int I = 2 * i, J = 2 * j;
  const int nodes[8][2] = {{0, 0}, {2, 0}, {0, 2}, {2, 2}, {1, 0}, {1, 2}, {0, 1}, {2, 1}};
  for (int n = 0; n < 8; ++n) {
    const Prim<T> w = L.at(I + nodes[n][0], J + nodes[n][1]);
    T o[4] = {T(0), T(0), T(0), T(0)};
    dcons_dprim_T(w, g, lU, n < 4 ? T(-0.0625) : T(-0.25), o);
    LA.add(I + nodes[n][0], J + nodes[n][1], o[0], o[1], o[2], o[3]);
  }
}

}  // namespace af
