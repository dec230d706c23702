// af_adjoint.cuh -- hand-written discrete adjoint of one step (Sec. 6.1):
// lambda^n = (d state^{n+1} / d state^n)^T lambda^{n+1}, linearised about the
// state at t^n.  The forward intermediates are recomputed by the unfused step
// kernels (af_ref_kernels.cuh); the reverse sweep then runs, one thread per
// cell, through
//   k_adj_flux      average update and space-time Simpson fluxes (gather)
//   k_adj_points    transported / additive point update, Q2 evaluation at the
//                   foot, the two Picard stages (all three point families)
//   k_adj_acoustic  Horner in r, node freezing (c, Z, r) and the transposed
//                   acoustic stencils (all four node families)
//   k_adj_center    Simpson inversion
// The scattering kernels add each contribution to global memory with one
// vector reduction: the adjoints of the lattice nodes and of the increments
// are kept as 4-wide records per node (FP32: one float4 atomic).  Adjoints are
// with respect to the stored variables; the storage offsets of the FP32 modes
// are constant shifts and do not change them.
#pragma once

#include "af_common.cuh"
#include "af_fused.cuh"
#include "af_launch.cuh"
#include "af_ref_kernels.cuh"

namespace af {

// Planes of one adjoint step, all with one stride (elements) from three bases.
template <typename T>
struct AdjView {
  const T* st;   // state^n: averages 0-3, points 4 + 4 fam + k
  const T* sto;  // state^{n+1} of the recomputed step: same layout
  const T* scr;  // intermediates: centres 0-3, increments 4 + 12 s + 3 fam + k,
                 // half-step points 28 + 4 fam + k
  T* lam;        // adjoints, in units of ps: lambda^{n+1} 0-15 and lambda^n of
                 // the averages 16-19 (planes); node records of family fam at
                 // 20 + 4 fam (4 values per cell: rho, u, v, p; family 3 is the
                 // centre); increment records of (s, fam) at 36 + 4 (4 s + fam)
                 // (du, dv, dp, 0); half- and full-step points 68 + 4 fam + k and
                 // 80 + 4 fam + k (planes); the centre adjoint lambda_U of each
                 // cell 92 + k (planes)
  size_t ps;
  int nx, ny;
  T h, dt;
  Gas<T> gas;
  int variant;
  const double* lin64[16];  // lambda^{n+1} as given (FP64 device planes), read by
                            // the fused reverse sweep in place of planes 0-15
};

constexpr int LAM_IN = 0, LAM_OUT = 16, LAM_NODE = 20, LAM_INC = 36, LAM_HALF = 68, LAM_FULL = 80;
constexpr int LAM_LU = 92;
constexpr int LAM_PLANES = 96;
constexpr int SCR_INC = 4, SCR_HALF = 28;

// family of lattice offset (a, b) from a cell's vertex: V, E_v, E_h, C
__host__ __device__ constexpr int fam_of(int a, int b) {
  return (a & 1) ? ((b & 1) ? 3 : 2) : ((b & 1) ? 1 : 0);
}

// cell index wrapped into [0, n): one conditional step for |i| < 2n
__device__ __forceinline__ int wrapc(int i, int n) {
  const int w = i < 0 ? i + n : (i >= n ? i - n : i);
  return (unsigned)w < (unsigned)n ? w : wrapi(i, n);
}

template <typename T>
__device__ __forceinline__ size_t cell_id(const AdjView<T>& v, int cx, int cy) {
  return (size_t)wrapc(cy, v.ny) * v.nx + wrapc(cx, v.nx);
}

// time-n value (rho~, u, v, p~) of the node of family fam of cell id
template <typename T>
__device__ __forceinline__ Prim<T> node_w(const AdjView<T>& v, int fam, size_t id) {
  const T* b = fam < 3 ? v.st + (size_t)(4 + 4 * fam) * v.ps : v.scr;
  Prim<T> w = {b[id], b[v.ps + id], b[2 * v.ps + id], b[3 * v.ps + id]};
  return w;
}

// increments (du, dv, dp) of duration s at the node of family fam of cell id
template <typename T>
__device__ __forceinline__ void node_d(const AdjView<T>& v, int s, int fam, size_t id, T d[3]) {
  const T* b = v.scr + (size_t)(SCR_INC + 12 * s + 3 * fam) * v.ps + id;
  d[0] = b[0];
  d[1] = b[v.ps];
  d[2] = b[2 * v.ps];
}

// Shared-memory accumulator over the footprint of a BX x BY block: cells
// [i0-1, i0+BX+2) x [j0-1, j0+BY+2), NPL planes; local plane lp < 16 is the
// adjoint of lattice plane 4 fam + k (global LAM_NODE + lp), lp >= 16 the
// adjoint of increment 12 s + 3 fam + k (global LAM_INC + lp - 16).
// adds (a, b, c, d) to the 4-wide record at p (16-byte aligned), without
// looking for zeros
__device__ __forceinline__ void add4_always(float* p, float a, float b, float c, float d) {
  atomicAdd(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
}
__device__ __forceinline__ void add4_always(double* p, double a, double b, double c, double d) {
  atomicAdd(p, a);
  atomicAdd(p + 1, b);
  atomicAdd(p + 2, c);
  atomicAdd(p + 3, d);
}

// clears the 4-wide record at p once its consumer has read it, so that the
// records start the next adjoint step at zero without a separate clearing pass
__device__ __forceinline__ void zero4(float* p) {
  *reinterpret_cast<float4*>(p) = make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void zero4(double* p) {
  reinterpret_cast<double2*>(p)[0] = make_double2(0.0, 0.0);
  reinterpret_cast<double2*>(p)[1] = make_double2(0.0, 0.0);
}

// adds (a, b, c, d) to the 4-wide record at p (16-byte aligned)
__device__ __forceinline__ void add4(float* p, float a, float b, float c, float d) {
  if (a != 0.f || b != 0.f || c != 0.f || d != 0.f)
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
}
__device__ __forceinline__ void add4(double* p, double a, double b, double c, double d) {
  if (a != 0.0) atomicAdd(p, a);
  if (b != 0.0) atomicAdd(p + 1, b);
  if (c != 0.0) atomicAdd(p + 2, c);
  if (d != 0.0) atomicAdd(p + 3, d);
}

// Accumulator of node and increment adjoints (records of the adjoint arena).
template <typename T>
struct VecAdj {
  T* lam;
  size_t ps;
  int nx, ny;
  __device__ __forceinline__ size_t cell(int cx, int cy) const {
    return (size_t)wrapc(cy, ny) * nx + wrapc(cx, nx);
  }
  // adjoint of the node of family fam of (unwrapped) cell (cx, cy)
  __device__ __forceinline__ void node(int fam, int cx, int cy, T r, T u, T w, T p) const {
    add4(lam + (size_t)(LAM_NODE + 4 * fam) * ps + 4 * cell(cx, cy), r, u, w, p);
  }
  __device__ __forceinline__ void inc(int s, int fam, int cx, int cy, T du, T dv, T dp) const {
    add4(lam + (size_t)(LAM_INC + 4 * (4 * s + fam)) * ps + 4 * cell(cx, cy), du, dv, dp, T(0));
  }
};

template <typename T>
__device__ __forceinline__ VecAdj<T> vec_adj(const AdjView<T>& v) {
  VecAdj<T> a = {v.lam, v.ps, v.nx, v.ny};
  return a;
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

// derivative of the Lagrange basis l_-, l_0, l_+ with respect to s
template <typename T>
__device__ __forceinline__ void lagrange3_d(T s, T d[3]) {
  d[0] = s - T(0.5);
  d[1] = T(-2) * s;
  d[2] = s + T(0.5);
}

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

template <int FAM, typename T, typename Scatter>
__device__ __forceinline__ void sac_family_adj(const Scatter& S, const T lGp[3][4],
                                               const T lGuv[3][4], T& lpK, T& luK, T& lvK) {
  if constexpr (FAM == 0) af_sac_V_adj<T>(S, lGp, lGuv, lpK, luK, lvK);
  if constexpr (FAM == 1) af_sac_EV_adj<T>(S, lGp, lGuv, lpK, luK, lvK);
  if constexpr (FAM == 2) af_sac_EH_adj<T>(S, lGp, lGuv, lpK, luK, lvK);
  if constexpr (FAM == 3) af_sac_C_adj<T>(S, lGp, lGuv, lpK, luK, lvK);
}


// ---------------------------------------------------------------------------
// Average update and fluxes (Eq. af-average-update), gathered per cell: the
// adjoints of the three point families of cell (i,j) at sigma = 0, 1/2, 1.
// Writes lambda^n of the averages and the sigma = 0 part of lambda^n of the
// points (the later kernels add to them), and the adjoints of the half- and
// full-step points.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ Prim<T> level_pt(const T* base, size_t ps, int f, size_t id) {
  const T* b = base + (size_t)(4 * f) * ps + id;
  Prim<T> w = {b[0], b[ps], b[2 * ps], b[3 * ps]};
  return w;
}

template <typename T>
__global__ void k_adj_flux(const __grid_constant__ AdjView<T> v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = v.nx, ny = v.ny;
  if (i >= nx || j >= ny) return;
  const size_t ps = v.ps;
  const int im = wrapc(i - 1, nx), jm = wrapc(j - 1, ny);
  const size_t id = (size_t)j * nx + i, idl = (size_t)j * nx + im, idb = (size_t)jm * nx + i,
               idlb = (size_t)jm * nx + im;
  T lfx[4], lfxb[4], lgy[4], lgyl[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T* lk = v.lam + (size_t)(LAM_IN + k) * ps;
    const T c = lk[id], l = lk[idl], b = lk[idb], lb = lk[idlb];
    lfx[k] = c - l;    // vertical edge x_i of cell (i,j)
    lfxb[k] = b - lb;  // vertical edge x_i of cell (i,j-1)
    lgy[k] = c - b;    // horizontal edge y_j of cell (i,j)
    lgyl[k] = l - lb;  // horizontal edge y_j of cell (i-1,j)
    v.lam[(size_t)(LAM_OUT + k) * ps + id] = c;
  }
  const T cst = v.dt / (T(36) * v.h);
  T lvx[4], lvy[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    lvx[k] = lfx[k] + lfxb[k];
    lvy[k] = lgy[k] + lgyl[k];
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    // point values at sigma = 0 (state^n), 1/2 (recomputed), 1 (state^{n+1})
    const T* base = s == 0 ? v.st + 4 * ps : s == 1 ? v.scr + (size_t)SCR_HALF * ps : v.sto + 4 * ps;
    const T sc = cst * (s == 1 ? T(4) : T(1));
    T oV[4] = {T(0), T(0), T(0), T(0)}, oEv[4] = {T(0), T(0), T(0), T(0)},
      oEh[4] = {T(0), T(0), T(0), T(0)};
    const Prim<T> wV = level_pt(base, ps, 0, id);
    flux_x_adj(wV, v.gas, lvx, sc, oV);
    flux_y_adj(wV, v.gas, lvy, sc, oV);
    flux_x_adj(level_pt(base, ps, 1, id), v.gas, lfx, T(4) * sc, oEv);
    flux_y_adj(level_pt(base, ps, 2, id), v.gas, lgy, T(4) * sc, oEh);
    const T* oo[3] = {oV, oEv, oEh};
    if (s == 0) {
      // lambda^n of the points starts as their node records (the later kernels add)
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        T* rec = v.lam + (size_t)(LAM_NODE + 4 * f) * ps + 4 * id;
#pragma unroll
        for (int k = 0; k < 4; ++k) rec[k] = oo[f][k];
      }
    } else {
      const int dst = s == 1 ? LAM_HALF : LAM_FULL;
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          T val = oo[f][k];
          if (s == 2) val += v.lam[(size_t)(LAM_IN + 4 + 4 * f + k) * ps + id];
          v.lam[(size_t)(dst + 4 * f + k) * ps + id] = val;
        }
    }
  }
}

// ---------------------------------------------------------------------------
// Point update (Sec. 6.1 steps 3-4; Eq. barsukow-additive), reversed.
// ---------------------------------------------------------------------------
// the nine nodes of foot cell c in [b][q] order (loaded once: the scatter
// below reuses them between its atomics)
template <typename T>
__device__ __forceinline__ void load_nodes(const AdjView<T>& v, const FootCell<T>& c, Prim<T> w[9]) {
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      w[3 * b + q] = node_w(v, fam_of(q, b), cell_id(v, c.ci + (q >> 1), c.cj + (b >> 1)));
}

template <typename T>
__device__ __forceinline__ void load_incs(const AdjView<T>& v, int s, const FootCell<T>& c,
                                          T d[9][3]) {
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      node_d(v, s, fam_of(q, b), cell_id(v, c.ci + (q >> 1), c.cj + (b >> 1)), d[3 * b + q]);
}

// sum_qb l_q(xi) l_b(eta) f_qb (rows first, as the forward evaluation)
template <typename T>
__device__ __forceinline__ T q2_sum(const T* f, int stride, const T lx[3], const T ly[3]) {
  T out = T(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    T row = T(0);
#pragma unroll
    for (int q = 0; q < 3; ++q) row = fma(lx[q], f[(3 * b + q) * stride], row);
    out = fma(ly[b], row, out);
  }
  return out;
}

// the point of family FAM of cell (i, j), both durations
template <int FAM, typename T, typename Acc>
__device__ __forceinline__ void point_adj(const AdjView<T>& v, const Acc& acc, int i, int j) {
  const size_t ps = v.ps, id = (size_t)j * v.nx + i;
  const int I = 2 * i + (FAM == 2 ? 1 : 0);
  const int J = 2 * j + (FAM == 1 ? 1 : 0);
  const Prim<T> wp = node_w(v, FAM, id);
  const T hinv = T(1) / v.h;
  const Gas<T>& g = v.gas;
  T luP = T(0), lvP = T(0), lrP = T(0), lpP = T(0);
#pragma unroll 1
  for (int s = 0; s < 2; ++s) {
    const T th = (s == 0 ? T(0.5) * v.dt : v.dt) * hinv;
    const T* lsrc = v.lam + (size_t)((s == 0 ? LAM_HALF : LAM_FULL) + 4 * FAM) * ps + id;
    const T ly[4] = {lsrc[0], lsrc[ps], lsrc[2 * ps], lsrc[3 * ps]};
    if (ly[0] == T(0) && ly[1] == T(0) && ly[2] == T(0) && ly[3] == T(0)) continue;
    // forward recomputation of the foot (Eq. adv-footpoint)
    const T d1x = -th * wp.u, d1y = -th * wp.v;
    const FootCell<T> c1 = locate<T>(I, J, d1x, d1y);
    T uv1[9][2];  // (u, v) of the first stage's nodes
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const Prim<T> w = node_w(v, fam_of(q, b), cell_id(v, c1.ci + (q >> 1), c1.cj + (b >> 1)));
        uv1[3 * b + q][0] = w.u;
        uv1[3 * b + q][1] = w.v;
      }
    T lx1[3], ly1[3];
    lagrange3(c1.xi, lx1);
    lagrange3(c1.eta, ly1);
    const T u1 = q2_sum(&uv1[0][0], 2, lx1, ly1), v1 = q2_sum(&uv1[0][1], 2, lx1, ly1);
    const T dfx = -th * u1, dfy = -th * v1;
    const FootCell<T> fc = locate<T>(I, J, dfx, dfy);
    Prim<T> nf[9];
    load_nodes(v, fc, nf);
    T lx[3], lyb[3], dx3[3], dy3[3];
    lagrange3(fc.xi, lx);
    lagrange3(fc.eta, lyb);
    lagrange3_d(fc.xi, dx3);
    lagrange3_d(fc.eta, dy3);
    Prim<T> wf;
    wf.r = q2_sum(&nf[0].r, 4, lx, lyb);
    wf.p = q2_sum(&nf[0].p, 4, lx, lyb);
    T lwf[4], ld[3];  // adjoints of W_f and of the interpolated increments
    T df[9][3];
    if (v.variant == 0) {
      load_incs(v, s, fc, df);
      const T d2 = q2_sum(&df[0][2], 3, lx, lyb);
      const T rf = g.rho_ref + wf.r, pf = g.p_ref + wf.p;
      const T gp = g.gamma * pf;
      lwf[0] = ly[0] * (T(1) + d2 / gp);
      lwf[1] = ly[1];
      lwf[2] = ly[2];
      lwf[3] = ly[3] - ly[0] * d2 * rf / (gp * pf);
      ld[0] = ly[1];
      ld[1] = ly[2];
      ld[2] = ly[3] + ly[0] * rf / gp;
    } else {
      T d[3];
      node_d(v, s, FAM, id, d);
      const T rp = g.rho_ref + wp.r, pp = g.p_ref + wp.p;
      const T gp = g.gamma * pp;
      lwf[0] = ly[0];
      lwf[1] = ly[1];
      lwf[2] = ly[2];
      lwf[3] = ly[3];
      // nw.r = wf.r + dp rho_P / (gamma p_P), with the increments at P itself
      acc.inc(s, FAM, i, j, ly[1], ly[2], ly[3] + ly[0] * rp / gp);
      lrP += ly[0] * d[2] / gp;
      lpP += -ly[0] * d[2] * rp / (gp * pp);
      ld[0] = ld[1] = ld[2] = T(0);
    }
    // adjoint of the foot's local coordinates through the Q2 evaluation there
    T lxi = T(0), leta = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int n = 3 * b + q;
        T dot = nf[n].r * lwf[0] + nf[n].u * lwf[1] + nf[n].v * lwf[2] + nf[n].p * lwf[3];
        if (v.variant == 0) dot += df[n][0] * ld[0] + df[n][1] * ld[1] + df[n][2] * ld[2];
        lxi += dx3[q] * lyb[b] * dot;
        leta += lx[q] * dy3[b] * dot;
      }
    // xi = 2 (foot - cell) - 1; the foot moved by df = -th (u1, v1)
    const T lu1 = -th * (T(2) * lxi), lv1 = -th * (T(2) * leta);
    // first Picard stage: (u1, v1) = R_h(u, v) at P + d1
    T dx31[3], dy31[3];
    lagrange3_d(c1.xi, dx31);
    lagrange3_d(c1.eta, dy31);
    T lxi1 = T(0), leta1 = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int n = 3 * b + q;
        const T dot = uv1[n][0] * lu1 + uv1[n][1] * lv1;
        lxi1 += dx31[q] * ly1[b] * dot;
        leta1 += lx1[q] * dy31[b] * dot;
      }
    luP += -th * (T(2) * lxi1);
    lvP += -th * (T(2) * leta1);
    // scatter to the nodes of the foot cell and of the first stage's cell (one
    // record update per node when the two cells coincide, the usual case)
    const bool same = c1.ci == fc.ci && c1.cj == fc.cj;
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int fam = fam_of(q, b), cx = fc.ci + (q >> 1), cy = fc.cj + (b >> 1);
        const T wgt = lx[q] * lyb[b], w1 = same ? lx1[q] * ly1[b] : T(0);
        acc.node(fam, cx, cy, wgt * lwf[0], wgt * lwf[1] + w1 * lu1, wgt * lwf[2] + w1 * lv1,
                 wgt * lwf[3]);
        if (v.variant == 0) acc.inc(s, fam, cx, cy, wgt * ld[0], wgt * ld[1], wgt * ld[2]);
      }
    if (!same) {
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const T w1 = lx1[q] * ly1[b];
          acc.node(fam_of(q, b), c1.ci + (q >> 1), c1.cj + (b >> 1), T(0), w1 * lu1, w1 * lv1,
                   T(0));
        }
    }
  }
  acc.node(FAM, i, j, lrP, luP, lvP, lpP);
}

template <int FAM, typename T>
__global__ void __launch_bounds__(256, 2) k_adj_points(const __grid_constant__ AdjView<T> v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i < v.nx && j < v.ny) point_adj<FAM>(v, vec_adj(v), i, j);
}

// ---------------------------------------------------------------------------
// Acoustic increments (Sec. 6.1 step 1), reversed: Horner in r_s = c tau_s / h,
// freezing c = sqrt(gamma p / rho), Z = rho c, and the transposed stencils.
// ---------------------------------------------------------------------------
// Wrapped neighbourhood of cell (ci, cj): columns ci-1, ci, ci+1 and row
// offsets (cj-1) nx, cj nx, (cj+1) nx; a lattice offset resolves at compile
// time to one of them.
struct Nbhd {
  int col[3];
  size_t row[3];
  __device__ __forceinline__ size_t at(int dc, int dr) const { return row[dr + 1] + col[dc + 1]; }
};

__device__ __forceinline__ Nbhd nbhd(int ci, int cj, int nx, int ny) {
  Nbhd b;
  b.col[1] = ci;
  b.col[0] = ci == 0 ? nx - 1 : ci - 1;
  b.col[2] = ci + 1 == nx ? 0 : ci + 1;
  const int rm = cj == 0 ? ny - 1 : cj - 1, rp = cj + 1 == ny ? 0 : cj + 1;
  b.row[0] = (size_t)rm * nx;
  b.row[1] = (size_t)cj * nx;
  b.row[2] = (size_t)rp * nx;
  return b;
}

// node values (.p, .u, .v) at lattice offset (dx, dy) from the node of family
// FAM of the neighbourhood's centre cell
template <int FAM, typename T>
struct LoadAdjPUV {
  const AdjView<T>* v;
  Nbhd b;
  __device__ __forceinline__ PUV<T> operator()(int dx, int dy) const {
    const int ax = ((FAM == 2 || FAM == 3) ? 1 : 0) + dx, by = ((FAM == 1 || FAM == 3) ? 1 : 0) + dy;
    const Prim<T> w = node_w(*v, fam_of(ax, by), b.at(ax >> 1, by >> 1));
    PUV<T> o = {w.p, w.u, w.v};
    return o;
  }
};

// adds (lp, lu, lv) to the record of the node at lattice offset (dx, dy).
// The warp is one row of consecutive nodes (lane = x offset); `act` holds the
// lanes taking part.  pair() takes a member (dx, dy), dx > 0, and its mirror
// (-dx, dy): the mirror's target seen from lane k + delta (delta = the cell
// distance between the two targets) is the member's target seen from lane k,
// so lane k adds lane k + delta's mirror values to its own and makes one
// record update for both; a mirror value whose lane k - delta is not taking
// part is added on its own.
template <int FAM, typename T>
struct ScatterAdj {
  T* lam;
  size_t ps;
  Nbhd b;
  unsigned act;
  __device__ __forceinline__ T* rec(int ax, int by) const {
    return lam + (size_t)(LAM_NODE + 4 * fam_of(ax, by)) * ps + 4 * b.at(ax >> 1, by >> 1);
  }
  __device__ __forceinline__ void operator()(int dx, int dy, T lp, T lu, T lv) const {
    constexpr int ox = (FAM == 2 || FAM == 3) ? 1 : 0, oy = (FAM == 1 || FAM == 3) ? 1 : 0;
    add4_always(rec(ox + dx, oy + dy), T(0), lu, lv, lp);
  }
  __device__ __forceinline__ void pair(int dx, int dy, T lp, T lu, T lv, T mp, T mu,
                                       T mv) const {
    constexpr int ox = (FAM == 2 || FAM == 3) ? 1 : 0, oy = (FAM == 1 || FAM == 3) ? 1 : 0;
    const int ax = ox + dx, am = ox - dx, by = oy + dy;
    const int delta = (ax >> 1) - (am >> 1);  // 1 or 2 (compile time once inlined)
    const int lane = threadIdx.x & 31;
    const T sp = __shfl_down_sync(act, mp, delta), su = __shfl_down_sync(act, mu, delta),
            sv = __shfl_down_sync(act, mv, delta);
    const bool take = lane + delta < 32 && ((act >> (lane + delta)) & 1u);
    const bool alone = lane < delta || !((act >> (lane - delta)) & 1u);
    add4_always(rec(ax, by), T(0), take ? lu + su : lu, take ? lv + sv : lv, take ? lp + sp : lp);
    if (alone) add4_always(rec(am, by), T(0), mu, mv, mp);
  }
  // members (2, dy), (-2, dy), (0, dy) of a family whose own column is even:
  // three consecutive nodes of one row, the right one lane k + 1's centre, the
  // left one lane k - 1's.  Each lane updates its centre with its neighbours'
  // right and left values, and its own right (left) value alone when lane
  // k + 1 (k - 1) is not taking part.
  __device__ __forceinline__ void triple(int dy, T rp, T ru, T rv, T lp, T lu, T lv, T cp, T cu,
                                         T cv) const {
    static_assert(FAM == 0 || FAM == 1, "the node's own column is even");
    constexpr int oy = FAM == 1 ? 1 : 0;
    const int by = oy + dy;
    const int lane = threadIdx.x & 31;
    const T ip = __shfl_up_sync(act, rp, 1), iu = __shfl_up_sync(act, ru, 1),
            iv = __shfl_up_sync(act, rv, 1);  // lane k - 1's right values
    const T jp = __shfl_down_sync(act, lp, 1), ju = __shfl_down_sync(act, lu, 1),
            jv = __shfl_down_sync(act, lv, 1);  // lane k + 1's left values
    const bool from_l = lane >= 1 && ((act >> (lane - 1)) & 1u);
    const bool from_r = lane <= 30 && ((act >> (lane + 1)) & 1u);
    T p = cp, u = cu, w = cv;
    if (from_l) {
      p += ip;
      u += iu;
      w += iv;
    }
    if (from_r) {
      p += jp;
      u += ju;
      w += jv;
    }
    add4_always(rec(0, by), T(0), u, w, p);
    if (!from_r) add4_always(rec(2, by), T(0), ru, rv, rp);
    if (!from_l) add4_always(rec(-2, by), T(0), lu, lv, lp);
  }
};

// `row`: the lanes of the calling warp (one row of 32 consecutive nodes) inside
// the grid
template <int FAM, typename T, typename Acc>
__device__ __forceinline__ void acoustic_adj(const AdjView<T>& v, const Acc& acc, int i, int j,
                                             unsigned row) {
  const size_t ps = v.ps, id = (size_t)j * v.nx + i;
  T ld[2][3];
  bool any = false;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    T* rec = v.lam + (size_t)(LAM_INC + 4 * (4 * s + FAM)) * ps + 4 * id;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ld[s][k] = rec[k];
      any = any || ld[s][k] != T(0);
    }
  }
  // the lanes of the row that have work: they take part in the merged scatter
  const unsigned act = __ballot_sync(row, any);
  if (!any) return;
#pragma unroll
  for (int s = 0; s < 2; ++s) zero4(v.lam + (size_t)(LAM_INC + 4 * (4 * s + FAM)) * ps + 4 * id);
  const Prim<T> wk = node_w(v, FAM, id);
  const T rk = v.gas.rho_ref + wk.r, pk = v.gas.p_ref + wk.p;
  const T c = sqrt(v.gas.gamma * pk / rk);
  const T Z = rk * c, Zinv = T(1) / Z;
  const T dth = v.dt / v.h;
  const T r1 = c * dth;
  T Gp[3][4], Guv[3][4];
  const Nbhd nb = nbhd(i, j, v.nx, v.ny);
  const LoadAdjPUV<FAM, T> ldr = {&v, nb};
  sac_family<FAM, T>(ldr, wk.p, wk.u, wk.v, Gp, Guv);
  // polynomial coefficients c_o[q] (q = 1..4 stored at 0..3), as in increments_at
  T co[3][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    co[2][q] = fma(Z, Guv[0][q], Gp[0][q]);     // dp
    co[0][q] = fma(Zinv, Gp[1][q], Guv[1][q]);  // du
    co[1][q] = fma(Zinv, Gp[2][q], Guv[2][q]);  // dv
  }
  T lco[3][4] = {}, lr1 = T(0);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T rs = s == 0 ? T(0.5) * r1 : r1;
    const T sc = s == 0 ? T(0.5) : T(1);
    T pw[5];
    pw[0] = T(1);
#pragma unroll
    for (int q = 1; q <= 4; ++q) pw[q] = pw[q - 1] * rs;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      T dr = T(0);
#pragma unroll
      for (int q = 1; q <= 4; ++q) {
        lco[o][q - 1] += pw[q] * ld[s][o];
        dr += T(q) * pw[q - 1] * co[o][q - 1];
      }
      lr1 += sc * dr * ld[s][o];
    }
  }
  T lGp[3][4], lGuv[3][4], lZ = T(0), lZinv = T(0);
#pragma unroll
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
  const T lrho = c * lZ - lc * c / (T(2) * rk);
  const T lp = lc * c / (T(2) * pk);
  T lpK = T(0), luK = T(0), lvK = T(0);
  const ScatterAdj<FAM, T> S = {v.lam, v.ps, nb, act};
  sac_family_adj<FAM, T>(S, lGp, lGuv, lpK, luK, lvK);
  acc.node(FAM, i, j, lrho, luK, lvK, lp + lpK);
}

// resident 256-thread blocks per SM requested of the acoustic and centre
// adjoints (their register budget follows; they wait on scattered loads)
#ifndef AF_ADJ_NODE_MINB
#define AF_ADJ_NODE_MINB 3
#endif

template <int FAM, typename T>
__global__ void __launch_bounds__(256, AF_ADJ_NODE_MINB)
    k_adj_acoustic(const __grid_constant__ AdjView<T> v) {
  // a warp is one row of 32 consecutive nodes (blockDim.x == 32)
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const unsigned row = __ballot_sync(0xffffffffu, i < v.nx && j < v.ny);
  if (i < v.nx && j < v.ny) acoustic_adj<FAM>(v, vec_adj(v), i, j, row);
}

// ---------------------------------------------------------------------------
// Centre recovery (Eq. center-node), reversed, in two parts: k_adj_center turns
// each cell's centre adjoint lambda_W into lambda_U (the adjoint of the
// recovered conserved centre), adds its 9/4 share to the cell average's lambda
// and stores lambda_U; k_adj_out then gives every vertex and edge node the
// -1/16 and -1/4 shares of the cells around it (a gather: four cells for a
// vertex, two for an edge, no atomics) before writing lambda^n out.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256, AF_ADJ_NODE_MINB)
    k_adj_center(const __grid_constant__ AdjView<T> v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const size_t ps = v.ps;
  if (i < v.nx && j < v.ny) {
    const size_t id = (size_t)j * v.nx + i;
    T* lc = v.lam + (size_t)(LAM_NODE + 12) * ps + 4 * id;  // the centre node's record
    const T lw[4] = {lc[0], lc[1], lc[2], lc[3]};
    T lU[4] = {T(0), T(0), T(0), T(0)};
    if (lw[0] != T(0) || lw[1] != T(0) || lw[2] != T(0) || lw[3] != T(0)) {
      zero4(lc);
      const Gas<T>& g = v.gas;
      // the recovered centre (rho~, u, v, p~) is W(U_c); lambda_U = (dW/dU)^T lambda_W
      const T rho = g.rho_ref + v.scr[id], u = v.scr[ps + id], w = v.scr[2 * ps + id];
      const T ri = T(1) / rho;
      lU[0] = lw[0] - u * ri * lw[1] - w * ri * lw[2] + g.gm1 * T(0.5) * (u * u + w * w) * lw[3];
      lU[1] = ri * lw[1] - g.gm1 * u * lw[3];
      lU[2] = ri * lw[2] - g.gm1 * w * lw[3];
      lU[3] = g.gm1 * lw[3];
      // U_c = 9/4 Ubar - 1/16 sum_corners U(W) - 1/4 sum_edges U(W); the
      // average of this cell has no other writer in this kernel
#pragma unroll
      for (int k = 0; k < 4; ++k) v.lam[(size_t)(LAM_OUT + k) * ps + id] += T(2.25) * lU[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) v.lam[(size_t)(LAM_LU + k) * ps + id] = lU[k];
  }
}

// ---------------------------------------------------------------------------
// Fused reverse sweep of a tile (FP32 modes).  fused_tile<..., ADJ> leaves the
// tile's time-n nodes W and the increments D of both durations in shared
// memory.  For each owned point: the adjoint of the space-time Simpson fluxes
// it enters (gathered from the averages' lambda, as k_adj_flux), then the
// adjoint of its point update for both durations (as k_adj_points) with the
// forward values taken from shared memory and the foot traced as the fused
// step traces it (displacements clamped to one cell).  Results go to the node
// and increment records (float4 atomics); the averages' lambda passes through.
// ---------------------------------------------------------------------------
template <int TX, int TY, int NT>
__device__ __forceinline__ void tile_reverse(const StepArgs<float>& a, const AdjView<float>& v,
                                             const float4* W, const float* D, int i0, int j0) {
  using G = FusedGeom<TX, TY>;
  constexpr int CW = G::CW, WPL = G::WPL, DCW = G::DCW, DPL = G::DPL;
  const int nx = a.nx, ny = a.ny;
  const size_t ps = v.ps;
  const Gas<float> gas = a.gas;
  const VecAdj<float> acc = vec_adj(v);
  const float th_full = a.dt / a.h;
  const float cst = a.dt / (36.f * a.h);
  static_assert(TX == 32 && (3 * TX * TY) % NT == 0, "a warp is one row of one family");
  const int lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < 3 * TX * TY; t += NT) {
    const int fam = t / (TX * TY), u = t - fam * (TX * TY);
    const int px = u % TX, py = u / TX;
    const int gi = i0 + px, gj = j0 + py;
    // lanes of the warp inside the grid (every lane of the warp is here)
    const unsigned mask = __ballot_sync(0xffffffffu, gi < nx && gj < ny);
    if (gi >= nx || gj >= ny) continue;
    const size_t id = (size_t)gj * nx + gi;
    // ---- fluxes (Eq. af-average-update), reversed ----
    const int im = wrapc(gi - 1, nx), jm = wrapc(gj - 1, ny);
    const size_t idl = (size_t)gj * nx + im, idb = (size_t)jm * nx + gi,
                 idlb = (size_t)jm * nx + im;
    float lex[4], ley[4];  // adjoints of the x- and y-fluxes the point enters
    if (fam == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double* lk = v.lin64[k];
        const float c = (float)lk[id], l = (float)lk[idl], b = (float)lk[idb],
                    lb = (float)lk[idlb];
        lex[k] = (c - l) + (b - lb);
        ley[k] = (c - b) + (l - lb);
        v.lam[(size_t)(LAM_OUT + k) * ps + id] = c;
      }
    } else if (fam == 1) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double* lk = v.lin64[k];
        lex[k] = (float)lk[id] - (float)lk[idl];
        ley[k] = 0.f;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double* lk = v.lin64[k];
        lex[k] = 0.f;
        ley[k] = (float)lk[id] - (float)lk[idb];
      }
    }
    const int wcP = (py + 2) * CW + (px + 2);
    const float4 wp = W[fam * WPL + wcP];
    float o0[4], lyh[4], lyf[4];  // sigma = 0 (own node), 1/2 and 1 (the point)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      Prim<float> w;
      if (s == 0) {
        w = prim4(wp);
      } else {
        float* const* src = s == 1 ? a.half[fam] : a.out.pt[fam];
        w.r = src[0][id];
        w.u = src[1][id];
        w.v = src[2][id];
        w.p = src[3][id];
      }
      const float sc = cst * (s == 1 ? 4.f : 1.f);
      float o[4] = {0.f, 0.f, 0.f, 0.f};
      if (fam == 0) {
        flux_x_adj(w, gas, lex, sc, o);
        flux_y_adj(w, gas, ley, sc, o);
      } else if (fam == 1) {
        flux_x_adj(w, gas, lex, 4.f * sc, o);
      } else {
        flux_y_adj(w, gas, ley, 4.f * sc, o);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (s == 0) o0[k] = o[k];
        else if (s == 1) lyh[k] = o[k];
        else lyf[k] = o[k] + (float)v.lin64[4 + 4 * fam + k][id];
      }
    }
    // ---- point update (Sec. 6.1 steps 3-4), reversed, both durations ----
    const int ox = fam == 2 ? 1 : 0, oy = fam == 1 ? 1 : 0;
    float luP = 0.f, lvP = 0.f, lrP = 0.f, lpP = 0.f;
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      const float th = s == 0 ? 0.5f * th_full : th_full;
      const float* Ds = D + s * 12 * DPL;
      float ly[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) ly[k] = s == 0 ? lyh[k] : lyf[k];
      // forward: the two Picard stages as the fused step traces them
      // (shared node records are (u, v, rho~, p~))
      const float d1x = clamp1(-th * wp.x), d1y = clamp1(-th * wp.y);
      float lx1[3], ly1[3];
      const int ix1 = foot_axis(ox, d1x, lx1), iy1 = foot_axis(oy, d1y, ly1);
      const int c1 = wcP + iy1 * CW + ix1;
      float4 n[9];
      load_cell<CW, WPL>(W, c1, n);
      const float u1 = AF_Q2(n, x, lx1, ly1), v1 = AF_Q2(n, y, lx1, ly1);
      const float dfx = clamp1(-th * u1), dfy = clamp1(-th * v1);
      float lx[3], lyb[3];
      const int ix = foot_axis(ox, dfx, lx), iy = foot_axis(oy, dfy, lyb);
      const int c2 = wcP + iy * CW + ix;
      if (c2 != c1) load_cell<CW, WPL>(W, c2, n);
      const float rft = AF_Q2(n, z, lx, lyb), pft = AF_Q2(n, w, lx, lyb);
      // local coordinates of the foot and of the first stage
      float dx3[3], dy3[3], dx31[3], dy31[3];
      {
        const float fx = fmaf(0.5f, (float)ox, dfx), fy = fmaf(0.5f, (float)oy, dfy);
        lagrange3_d(fmaf(2.f, fx - floorf(fx), -1.f), dx3);
        lagrange3_d(fmaf(2.f, fy - floorf(fy), -1.f), dy3);
        const float gx = fmaf(0.5f, (float)ox, d1x), gy = fmaf(0.5f, (float)oy, d1y);
        lagrange3_d(fmaf(2.f, gx - floorf(gx), -1.f), dx31);
        lagrange3_d(fmaf(2.f, gy - floorf(gy), -1.f), dy31);
      }
      const int dcf = (py + 1 + iy) * DCW + (px + 1 + ix);  // D cell of the foot cell
      float lwf[4], ld[3];  // adjoints of W at the foot and of the interpolated increments
      if (a.variant == 0) {
        const float d2 = q2_eval<DCW>(Ds + 2 * DPL, Ds + 5 * DPL, Ds + 8 * DPL, Ds + 11 * DPL,
                                      dcf, lx, lyb);
        // (fast reciprocals, as the forward closure's division)
        const float rf = gas.rho_ref + rft, pf = gas.p_ref + pft;
        const float igp = __fdividef(1.f, gas.gamma * pf), ipf = __fdividef(1.f, pf);
        lwf[0] = ly[0] * fmaf(d2, igp, 1.f);
        lwf[1] = ly[1];
        lwf[2] = ly[2];
        lwf[3] = ly[3] - ly[0] * d2 * rf * igp * ipf;
        ld[0] = ly[1];
        ld[1] = ly[2];
        ld[2] = fmaf(ly[0] * rf, igp, ly[3]);
      } else {
        const int dcp = (py + 1) * DCW + (px + 1);
        const float d2 = Ds[(fam * 3 + 2) * DPL + dcp];
        const float rp = gas.rho_ref + wp.z, pp = gas.p_ref + wp.w;
        const float igp = __fdividef(1.f, gas.gamma * pp), ipp = __fdividef(1.f, pp);
#pragma unroll
        for (int k = 0; k < 4; ++k) lwf[k] = ly[k];
        // rho = rho_f + dp rho_P / (gamma p_P), with the increments at P itself
        acc.inc(s, fam, gi, gj, ly[1], ly[2], fmaf(ly[0] * rp, igp, ly[3]));
        lrP += ly[0] * d2 * igp;
        lpP += -ly[0] * d2 * rp * igp * ipp;
        ld[0] = ld[1] = ld[2] = 0.f;
      }
      // adjoint of the foot's local coordinates.  D holds (u + du, v + dv) and dp;
      // u and du enter the transported update with the same weight.
      float lxi = 0.f, leta = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int m = 3 * b + q, fn = fam_of(q, b);
          float dot;
          if (a.variant == 0) {
            const int dn = dcf + (b >> 1) * DCW + (q >> 1);
            const float2 uv = reinterpret_cast<const float2*>(Ds + fn * 3 * DPL)[dn];
            dot = n[m].z * lwf[0] + uv.x * lwf[1] + uv.y * lwf[2] + n[m].w * lwf[3] +
                  Ds[(fn * 3 + 2) * DPL + dn] * ld[2];
          } else {
            dot = n[m].z * lwf[0] + n[m].x * lwf[1] + n[m].y * lwf[2] + n[m].w * lwf[3];
          }
          lxi += dx3[q] * lyb[b] * dot;
          leta += lx[q] * dy3[b] * dot;
        }
      // xi = 2 (foot - cell) - 1; the foot moved by df = -th (u1, v1)
      const float lu1 = -th * (2.f * lxi), lv1 = -th * (2.f * leta);
      // first Picard stage: (u1, v1) = R_h(u, v) at P + d1
      if (c2 != c1) load_cell<CW, WPL>(W, c1, n);
      float lxi1 = 0.f, leta1 = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int m = 3 * b + q;
          const float dot = n[m].x * lu1 + n[m].y * lv1;
          lxi1 += dx31[q] * ly1[b] * dot;
          leta1 += lx1[q] * dy31[b] * dot;
        }
      luP += -th * (2.f * lxi1);
      lvP += -th * (2.f * leta1);
      // scatter to the foot cell's nodes (and the first stage's, merged when
      // both use the same cell).  When the right-hand neighbour lane (the next
      // point of the row) has its foot at the same offset, its first node
      // column is this lane's last: it hands those contributions over and this
      // lane adds them with its own (one record update instead of two).
      const bool same = c1 == c2;
      // wrapped cells of the foot cell's 2 x 2 block of node cells
      const int col0 = wrapc(gi + ix, nx), col1 = col0 + 1 == nx ? 0 : col0 + 1;
      const size_t row0 = (size_t)wrapc(gj + iy, ny) * nx;
      const size_t row1 = (row0 + nx == (size_t)ny * nx) ? 0 : row0 + nx;
      const int key = (ix + 2) + 8 * (iy + 2);
      const int lkey = __shfl_up_sync(mask, key, 1), rkey = __shfl_down_sync(mask, key, 1);
      const bool give = lane > 0 && ((mask >> (lane - 1)) & 1u) && lkey == key;
      const bool take = lane < 31 && ((mask >> (lane + 1)) & 1u) && rkey == key;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        float nd[3][4], ic[3][3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float wgt = lx[q] * lyb[b], w1 = same ? lx1[q] * ly1[b] : 0.f;
          nd[q][0] = wgt * lwf[0];
          nd[q][1] = fmaf(w1, lu1, wgt * lwf[1]);
          nd[q][2] = fmaf(w1, lv1, wgt * lwf[2]);
          nd[q][3] = wgt * lwf[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) ic[q][k] = wgt * ld[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float r = __shfl_down_sync(mask, nd[0][k], 1);
          if (take) nd[2][k] += r;
        }
        if (a.variant == 0) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float r = __shfl_down_sync(mask, ic[0][k], 1);
            if (take) ic[2][k] += r;
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (q == 0 && give) continue;
          const int fn = fam_of(q, b);
          const size_t cell = (b >> 1 ? row1 : row0) + (q >> 1 ? col1 : col0);
          float* nr = v.lam + (size_t)(LAM_NODE + 4 * fn) * ps + 4 * cell;
          atomicAdd(reinterpret_cast<float4*>(nr),
                    make_float4(nd[q][0], nd[q][1], nd[q][2], nd[q][3]));
          if (a.variant == 0) {
            float* ir = v.lam + (size_t)(LAM_INC + 4 * (4 * s + fn)) * ps + 4 * cell;
            atomicAdd(reinterpret_cast<float4*>(ir),
                      make_float4(ic[q][0], ic[q][1], ic[q][2], 0.f));
          }
        }
      }
      if (!same) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float w1 = lx1[q] * ly1[b];
            acc.node(fam_of(q, b), gi + ix1 + (q >> 1), gj + iy1 + (b >> 1), 0.f, w1 * lu1,
                     w1 * lv1, 0.f);
          }
      }
    }
    acc.node(fam, gi, gj, o0[0] + lrP, o0[1] + luP, o0[2] + lvP, o0[3] + lpP);
  }
}

// Persistent kernel of the fused reverse sweep: the pipelined step's tile loop
// (k_fused_step_pipe) with fused_tile<..., ADJ> and tile_reverse per tile; the
// next tile's input is staged once the reverse sweep is done with D.
template <int TX, int TY, int NT, int MINB, bool COMP>
__global__ void __launch_bounds__(NT, MINB)
    k_fused_adj_pipe(const __grid_constant__ StepArgs<float> a, const __grid_constant__ TileMaps tm,
                     int use_tma, const __grid_constant__ AdjView<float> v) {
  using G = FusedGeom<TX, TY>;
  extern __shared__ __align__(16) float4 smem4[];
  float* S = reinterpret_cast<float*>(smem4 + 4 * G::WPL);
  PipeCtx pc;
  pc.tm = (use_tma && G::W_BYTES % 128 == 0 && (smem_addr(smem4) & 127u) == 0) ? &tm : nullptr;
  pc.bar = smem_addr(reinterpret_cast<char*>(smem4) + G::SMEM);
  pc.phase = 0;
  pc.late = 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pc.bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int tcols = (a.nx + TX - 1) / TX, ntiles = tcols * ((a.ny + TY - 1) / TY);
  int tile = blockIdx.x;
  if (tile < ntiles)
    issue_tile_async<TX, TY, NT, COMP>(a, pc, (tile % tcols) * TX, (tile / tcols) * TY, S);
  for (; tile < ntiles; tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    const int pi0 = nxt < ntiles ? (nxt % tcols) * TX : -1, pj0 = (nxt / tcols) * TY;
    const int i0 = (tile % tcols) * TX, j0 = (tile / tcols) * TY;
    if (!fused_tile<TX, TY, NT, COMP, true, false, true>(a, pc, i0, j0, pi0, pj0,
                                                         a.prefetch_wave > 0 && !pc.tm))
      break;
    tile_reverse<TX, TY, NT>(a, v, smem4, S, i0, j0);
    __syncthreads();  // W and D are dead from here
    if (pi0 >= 0) issue_tile_async<TX, TY, NT, COMP>(a, pc, pi0, pj0, S);
  }
}

// Launches the fused reverse sweep when the pipelined kernel accepts the grid
// (cudaErrorNotSupported otherwise).
template <bool COMP>
inline cudaError_t launch_fused_adjoint(cudaStream_t s, const StepArgs<float>& a, int ctas,
                                        const TileMaps* maps, const AdjView<float>& v) {
  using G = FusedGeom<FUSED_TX, FUSED_TY>;
  if (!(ctas > 0 && pipe_eligible(a))) return cudaErrorNotSupported;
  constexpr auto kern = k_fused_adj_pipe<FUSED_TX, FUSED_TY, FUSED_NT, AF_FUSED_MINB, COMP>;
  const cudaError_t e = allow_smem<kern>(G::SMEM_PIPE);
  if (e != cudaSuccess) return e;
  static TileMaps none;
  const int ntiles = ((a.nx + FUSED_TX - 1) / FUSED_TX) * ((a.ny + FUSED_TY - 1) / FUSED_TY);
  kern<<<ntiles < ctas ? ntiles : ctas, FUSED_NT, G::SMEM_PIPE, s>>>(a, maps ? *maps : none,
                                                                       maps ? 1 : 0, v);
  return cudaGetLastError();
}

// Sixteen planes converted in one launch (the adjoint state in and out).
template <typename A, typename B>
struct Cast16 {
  const A* src[16];
  B* dst[16];
};

template <typename A, typename B>
__global__ void k_cast16(const __grid_constant__ Cast16<A, B> c, size_t n) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int p = 0; p < 16; ++p) c.dst[p][t] = (B)c.src[p][t];
  }
}

// lambda^n out: the averages' planes and the point families' node records into
// sixteen FP64 planes
template <typename T>
struct AdjOut {
  double* dst[16];
};

template <typename T>
__global__ void k_adj_out(const __grid_constant__ AdjView<T> v,
                          const __grid_constant__ AdjOut<T> o, size_t n) {
  const size_t ps = v.ps;
  const Gas<T>& g = v.gas;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 4; ++k) o.dst[k][t] = (double)v.lam[(size_t)(LAM_OUT + k) * ps + t];
    // lambda_U of the cells around this cell's vertex (i, j): (i, j), (i-1, j),
    // (i, j-1), (i-1, j-1); the x-edge (i+1/2, j) lies in (i, j) and (i, j-1),
    // the y-edge (i, j+1/2) in (i, j) and (i-1, j)
    const int j = (int)(t / (size_t)v.nx), i = (int)(t - (size_t)j * v.nx);
    const size_t il = (size_t)j * v.nx + wrapc(i - 1, v.nx);
    const size_t jb = (size_t)wrapc(j - 1, v.ny) * v.nx;
    const size_t ib = jb + i, ilb = jb + wrapc(i - 1, v.nx);
    T lc[4], ll[4], lb[4], llb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T* pl = v.lam + (size_t)(LAM_LU + k) * ps;
      lc[k] = pl[t];
      ll[k] = pl[il];
      lb[k] = pl[ib];
      llb[k] = pl[ilb];
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      T* rec = v.lam + (size_t)(LAM_NODE + 4 * f) * ps + 4 * t;
      T r[4] = {rec[0], rec[1], rec[2], rec[3]}, sum[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        sum[k] = f == 0 ? (lc[k] + ll[k]) + (lb[k] + llb[k]) : (f == 1 ? lc[k] + ll[k] : lc[k] + lb[k]);
      dcons_dprim_T(node_w(v, f, t), g, sum, f == 0 ? T(-0.0625) : T(-0.25), r);
#pragma unroll
      for (int k = 0; k < 4; ++k) o.dst[4 + 4 * f + k][t] = (double)r[k];
      zero4(rec);
    }
  }
}

}  // namespace af
