// af_ref_kernels.cuh -- the RB-TAI / RB step as separate simple kernels, one
// thread per cell, intermediate values in global scratch.  It is the FP64
// path and the reference layout for the fused kernel:
//   k_center    centre recovery by Simpson inversion        (Eq. center-node)
//   k_acoustic  node-centred exact acoustic increments      (Sec. 6.1 step 1)
//   k_points    two-Picard foot + transported / additive    (Sec. 6.1 steps 2-4,
//               point update at tau = dt/2 and dt           Eq. barsukow-additive)
//   k_flux      space-time Simpson edge fluxes              (Sec. 3.1, Sec. 6.1)
//   k_average   conservative average update                 (Eq. af-average-update)
#pragma once

#include "af_common.cuh"
#include "af_stencils.cuh"

namespace af {

template <typename T>
struct StepArgs {
  Planes<T> in;       // state at t^n
  Planes<T> out;      // state at t^{n+1}
  T* wc[4];           // recovered centre (rho, u, v, p)
  T* inc[2][4][3];    // [tau index][family V,Ev,Eh,C][du, dv, dp]
  T* half[3][4];      // point values at t^n + dt/2, [family][rho,u,v,p]
  T* fx[4];           // (dt/h) * time-integrated flux through vertical edge (i,j)
  T* gy[4];           // (dt/h) * time-integrated flux through horizontal edge (i,j)
  unsigned* flags;
  int nx, ny;
  T h, dt;
  Gas<T> gas;
  int variant;        // 0 TAI, 1 RB
  int prefetch_wave;  // fused kernel: blocks per wave for the L2 prefetch (0: none)
  int late_first_wait;  // pipelined kernels, testing only: each CTA's first wait for a
                        // tensor-copied tile reports a timeout at once (0: off)
};

template <typename T>
__device__ __forceinline__ LatticeG<T> lattice_of(const StepArgs<T>& a) {
  LatticeG<T> L;
  for (int f = 0; f < 3; ++f)
    for (int k = 0; k < 4; ++k) L.f[f][k] = a.in.pt[f][k];
  for (int k = 0; k < 4; ++k) L.f[3][k] = a.wc[k];
  L.nx = a.nx;
  L.ny = a.ny;
  return L;
}

__device__ __forceinline__ void raise_flag(unsigned* flags, unsigned bits) {
  if (bits) atomicOr(flags, bits);
}

// ---------------------------------------------------------------------------
// Centre recovery (Eq. center-node) in the algebraically equal deviation form
// U_c = Ubar + 1/16 sum_corners (Ubar - U_V) + 1/4 sum_edges (Ubar - U_E).
// ---------------------------------------------------------------------------
template <typename T, bool COMP>
__global__ void k_center(StepArgs<T> a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  int ip = wrapi(i + 1, a.nx), jp = wrapi(j + 1, a.ny);
  size_t id = (size_t)j * a.nx + i;
  auto P = [&](int f, int ii, int jj) {
    size_t q = (size_t)jj * a.nx + ii;
    Prim<T> w = {a.in.pt[f][0][q], a.in.pt[f][1][q], a.in.pt[f][2][q], a.in.pt[f][3][q]};
    return w;
  };
  T ub[4], lo[4], uc[4], c[4], e[4];
  for (int k = 0; k < 4; ++k) {
    ub[k] = a.in.avg[k][id];
    lo[k] = COMP ? a.in.lo[k][id] : T(0);
    c[k] = T(0);
    e[k] = T(0);
  }
  const Prim<T> corners[4] = {P(0, i, j), P(0, ip, j), P(0, i, jp), P(0, ip, jp)};
  const Prim<T> edges[4] = {P(2, i, j), P(2, i, jp), P(1, i, j), P(1, ip, j)};
  for (int n = 0; n < 4; ++n) {
    T u[4];
    cons_from_stored(corners[n], a.gas, u);
    for (int k = 0; k < 4; ++k) c[k] += (ub[k] - u[k]) + lo[k];
    cons_from_stored(edges[n], a.gas, u);
    for (int k = 0; k < 4; ++k) e[k] += (ub[k] - u[k]) + lo[k];
  }
  for (int k = 0; k < 4; ++k) uc[k] = (ub[k] + lo[k]) + (T(0.0625) * c[k] + T(0.25) * e[k]);
  Prim<T> w = stored_from_cons(uc, a.gas);
  a.wc[0][id] = w.r;
  a.wc[1][id] = w.u;
  a.wc[2][id] = w.v;
  a.wc[3][id] = w.p;
  raise_flag(a.flags, (a.gas.rho_ref + w.r > T(0) && a.gas.p_ref + w.p > T(0)) ? 0u
                                                                             : FLAG_NONPHYSICAL);
}

// ---------------------------------------------------------------------------
// Exact frozen acoustic increments at the nodes of one family, for tau = dt/2
// and tau = dt (Sec. 6.1 step 1).  The r^q sums are shared by both durations.
// ---------------------------------------------------------------------------
template <typename T>
struct LoadPUV {
  const LatticeG<T>* L;
  int I, J;
  __device__ __forceinline__ PUV<T> operator()(int dx, int dy) const {
    Prim<T> w = L->at(I + dx, J + dy);
    PUV<T> o = {w.p, w.u, w.v};
    return o;
  }
};

template <int FAM, typename T, typename Load>
__device__ __forceinline__ void sac_family(const Load& L, T pK, T uK, T vK, T Gp[3][4],
                                           T Guv[3][4]) {
  if (FAM == 0) af_sac_V<T>(L, pK, uK, vK, Gp, Guv);
  if (FAM == 1) af_sac_EV<T>(L, pK, uK, vK, Gp, Guv);
  if (FAM == 2) af_sac_EH<T>(L, pK, uK, vK, Gp, Guv);
  if (FAM == 3) af_sac_C<T>(L, pK, uK, vK, Gp, Guv);
}

// Horner evaluation of the increments: dp = sum_q r^q (Gp0 + Z Guv0), etc.
template <typename T>
__device__ __forceinline__ void increments_at(const T Gp[3][4], const T Guv[3][4], T Z, T Zinv,
                                              T r, T d[3]) {
  T cp[4], cu[4], cv[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    cp[q] = fma(Z, Guv[0][q], Gp[0][q]);
    cu[q] = fma(Zinv, Gp[1][q], Guv[1][q]);
    cv[q] = fma(Zinv, Gp[2][q], Guv[2][q]);
  }
  d[2] = r * fma(r, fma(r, fma(r, cp[3], cp[2]), cp[1]), cp[0]);
  d[0] = r * fma(r, fma(r, fma(r, cu[3], cu[2]), cu[1]), cu[0]);
  d[1] = r * fma(r, fma(r, fma(r, cv[3], cv[2]), cv[1]), cv[0]);
}

template <int FAM, typename T>
__global__ void k_acoustic(StepArgs<T> a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  LatticeG<T> L = lattice_of(a);
  const int I = 2 * i + ((FAM == 2 || FAM == 3) ? 1 : 0);
  const int J = 2 * j + ((FAM == 1 || FAM == 3) ? 1 : 0);
  Prim<T> wk = L.at(I, J);
  unsigned bad = 0;
  const T rk = a.gas.rho_ref + wk.r, pk = a.gas.p_ref + wk.p;
  if (!(rk > T(0) && pk > T(0))) bad |= FLAG_NONPHYSICAL;
  T c = sqrt(a.gas.gamma * pk / rk);
  T Z = rk * c, Zinv = T(1) / Z;
  T r1 = c * a.dt / a.h;
  if (r1 > T(0.5)) bad |= FLAG_CFL;
  T Gp[3][4], Guv[3][4];
  LoadPUV<T> ld = {&L, I, J};
  sac_family<FAM, T>(ld, wk.p, wk.u, wk.v, Gp, Guv);
  size_t id = (size_t)j * a.nx + i;
  for (int s = 0; s < 2; ++s) {
    T d[3];
    increments_at(Gp, Guv, Z, Zinv, s == 0 ? T(0.5) * r1 : r1, d);
    a.inc[s][FAM][0][id] = d[0];
    a.inc[s][FAM][1][id] = d[1];
    a.inc[s][FAM][2][id] = d[2];
  }
  raise_flag(a.flags, bad);
}

// ---------------------------------------------------------------------------
// Point update (Sec. 6.1 steps 3-4).  Positions are kept as an integer cell
// index plus a small offset so that FP32 resolves the foot on large grids.
// ---------------------------------------------------------------------------
template <typename T>
struct FootCell {
  int ci, cj;  // cell containing the point
  T xi, eta;   // local coordinates in [-1, 1]
};

// point at lattice (I, J) displaced by (dx, dy) cells
template <typename T>
__device__ __forceinline__ FootCell<T> locate(int I, int J, T dx, T dy) {
  T fx = T(0.5) * (T)(I & 1) + dx;
  T fy = T(0.5) * (T)(J & 1) + dy;
  T flx = floor(fx), fly = floor(fy);
  FootCell<T> c;
  c.ci = (I >> 1) + (int)flx;
  c.cj = (J >> 1) + (int)fly;
  c.xi = T(2) * (fx - flx) - T(1);
  c.eta = T(2) * (fy - fly) - T(1);
  return c;
}

template <typename T>
__device__ __forceinline__ Prim<T> eval_w(const LatticeG<T>& L, const FootCell<T>& c) {
  T lx[3], ly[3];
  lagrange3(c.xi, lx);
  lagrange3(c.eta, ly);
  Prim<T> s = {T(0), T(0), T(0), T(0)};
  for (int b = 0; b < 3; ++b) {
    Prim<T> row = {T(0), T(0), T(0), T(0)};
    for (int q = 0; q < 3; ++q) {
      Prim<T> w = L.at(2 * c.ci + q, 2 * c.cj + b);
      row.r = fma(lx[q], w.r, row.r);
      row.u = fma(lx[q], w.u, row.u);
      row.v = fma(lx[q], w.v, row.v);
      row.p = fma(lx[q], w.p, row.p);
    }
    s.r = fma(ly[b], row.r, s.r);
    s.u = fma(ly[b], row.u, s.u);
    s.v = fma(ly[b], row.v, s.v);
    s.p = fma(ly[b], row.p, s.p);
  }
  return s;
}

template <typename T>
__device__ __forceinline__ void eval_d(const IncrG<T>& D, const FootCell<T>& c, T out[3]) {
  T lx[3], ly[3];
  lagrange3(c.xi, lx);
  lagrange3(c.eta, ly);
  out[0] = out[1] = out[2] = T(0);
  for (int b = 0; b < 3; ++b) {
    T row[3] = {T(0), T(0), T(0)};
    for (int q = 0; q < 3; ++q) {
      T d[3];
      D.at(2 * c.ci + q, 2 * c.cj + b, d);
      for (int k = 0; k < 3; ++k) row[k] = fma(lx[q], d[k], row[k]);
    }
    for (int k = 0; k < 3; ++k) out[k] = fma(ly[b], row[k], out[k]);
  }
}

template <int FAM, typename T>
__global__ void k_points(StepArgs<T> a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  LatticeG<T> L = lattice_of(a);
  const int I = 2 * i + (FAM == 2 ? 1 : 0);
  const int J = 2 * j + (FAM == 1 ? 1 : 0);
  const Prim<T> wp = L.at(I, J);
  const T hinv = T(1) / a.h;
  size_t id = (size_t)j * a.nx + i;
  unsigned bad = 0;
  for (int s = 0; s < 2; ++s) {
    const T tau = s == 0 ? T(0.5) * a.dt : a.dt;
    const T th = tau * hinv;
    IncrG<T> D;
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < 3; ++k) D.f[f][k] = a.inc[s][f][k];
    D.nx = a.nx;
    D.ny = a.ny;
    // two-Picard convective foot from the time-n reconstruction (Eq. adv-footpoint)
    T d1x = -th * wp.u, d1y = -th * wp.v;
    Prim<T> w1 = eval_w(L, locate<T>(I, J, d1x, d1y));
    T dfx = -th * w1.u, dfy = -th * w1.v;
    if (fabs(d1x) > T(1) || fabs(d1y) > T(1) || fabs(dfx) > T(1) || fabs(dfy) > T(1))
      bad |= FLAG_REACH;
    FootCell<T> fc = locate<T>(I, J, dfx, dfy);
    Prim<T> wf = eval_w(L, fc);
    Prim<T> nw;
    if (a.variant == 0) {
      // transported increment evaluated at the foot; rho from dp / c_f^2
      T d[3];
      eval_d(D, fc, d);
      const T rf = a.gas.rho_ref + wf.r, pf = a.gas.p_ref + wf.p;
      if (!(rf > T(0) && pf > T(0))) bad |= FLAG_NONPHYSICAL;
      nw.r = wf.r + d[2] * rf / (a.gas.gamma * pf);
      nw.u = wf.u + d[0];
      nw.v = wf.v + d[1];
      nw.p = wf.p + d[2];
    } else {
      // additive update: S_ac(P) + S_adv(P) - W(P), acoustic rho closure at P
      T d[3];
      D.at(I, J, d);
      nw.r = wf.r + d[2] * (a.gas.rho_ref + wp.r) / (a.gas.gamma * (a.gas.p_ref + wp.p));
      nw.u = wf.u + d[0];
      nw.v = wf.v + d[1];
      nw.p = wf.p + d[2];
    }
    if (!(isfinite(nw.r) && isfinite(nw.u) && isfinite(nw.v) && isfinite(nw.p)))
      bad |= FLAG_NONFINITE;
    T* const* dst = s == 0 ? a.half[FAM] : a.out.pt[FAM];
    dst[0][id] = nw.r;
    dst[1][id] = nw.u;
    dst[2][id] = nw.v;
    dst[3][id] = nw.p;
  }
  raise_flag(a.flags, bad);
}

// ---------------------------------------------------------------------------
// Space-time Simpson fluxes (Sec. 3.1, Sec. 6.1), scaled by dt/h.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ Prim<T> load_pt(T* const* pl, size_t q) {
  Prim<T> w = {pl[0][q], pl[1][q], pl[2][q], pl[3][q]};
  return w;
}

template <typename T>
__global__ void k_flux(StepArgs<T> a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  size_t id = (size_t)j * a.nx + i;
  size_t up = (size_t)wrapi(j + 1, a.ny) * a.nx + i;
  size_t rt = (size_t)j * a.nx + wrapi(i + 1, a.nx);
  T* const* lev[3][3] = {{a.in.pt[0], a.in.pt[1], a.in.pt[2]},
                         {a.half[0], a.half[1], a.half[2]},
                         {a.out.pt[0], a.out.pt[1], a.out.pt[2]}};
  const T wt[3] = {T(1), T(4), T(1)};
  T F[4] = {T(0), T(0), T(0), T(0)}, G[4] = {T(0), T(0), T(0), T(0)};
  for (int s = 0; s < 3; ++s) {
    T fa[4], fm[4], fb[4];
    // vertical edge x = x_i: V(i,j), E_v(i,j), V(i,j+1)
    flux_x(load_pt<T>(lev[s][0], id), a.gas, fa);
    flux_x(load_pt<T>(lev[s][1], id), a.gas, fm);
    flux_x(load_pt<T>(lev[s][0], up), a.gas, fb);
    for (int k = 0; k < 4; ++k) F[k] = fma(wt[s], fa[k] + T(4) * fm[k] + fb[k], F[k]);
    // horizontal edge y = y_j: V(i,j), E_h(i,j), V(i+1,j)
    flux_y(load_pt<T>(lev[s][0], id), a.gas, fa);
    flux_y(load_pt<T>(lev[s][2], id), a.gas, fm);
    flux_y(load_pt<T>(lev[s][0], rt), a.gas, fb);
    for (int k = 0; k < 4; ++k) G[k] = fma(wt[s], fa[k] + T(4) * fm[k] + fb[k], G[k]);
  }
  const T lam = a.dt / (T(36) * a.h);
  for (int k = 0; k < 4; ++k) {
    a.fx[k][id] = lam * F[k];
    a.gy[k][id] = lam * G[k];
  }
}

// Conservative average update (Eq. af-average-update).  COMP: hi + lo pairs
// updated by error-free sums of the four edge terms, so that each edge value
// enters its two cells with opposite signs exactly.
template <typename T, bool COMP>
__global__ void k_average(StepArgs<T> a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  size_t id = (size_t)j * a.nx + i;
  size_t up = (size_t)wrapi(j + 1, a.ny) * a.nx + i;
  size_t rt = (size_t)j * a.nx + wrapi(i + 1, a.nx);
  unsigned bad = 0;
  for (int k = 0; k < 4; ++k) {
    if constexpr (COMP) {
      float hi = a.in.avg[k][id], lo = a.in.lo[k][id];
      comp_update(hi, lo, a.fx[k][id], a.fx[k][rt], a.gy[k][id], a.gy[k][up]);
      a.out.avg[k][id] = hi;
      a.out.lo[k][id] = lo;
      if (!isfinite(hi)) bad |= FLAG_NONFINITE;
    } else {
      T v = a.in.avg[k][id] - (a.fx[k][rt] - a.fx[k][id]) - (a.gy[k][up] - a.gy[k][id]);
      a.out.avg[k][id] = v;
      if (!isfinite(v)) bad |= FLAG_NONFINITE;
    }
  }
  raise_flag(a.flags, bad);
}

}  // namespace af
