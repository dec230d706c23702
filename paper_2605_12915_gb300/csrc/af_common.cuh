// af_common.cuh -- device building blocks shared by the kernels of the RB-TAI
// Active Flux step: gas model (Sec. 2), Q2 Lagrange basis (Sec. 4), the
// half-cell lattice addressing of the point values, error bits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace af {

// device error bits (latched with atomicOr; mapped to af_status on the host)
enum : unsigned {
  FLAG_CFL = 1u,          // c_K dt / h > 1/2 at a node
  FLAG_NONPHYSICAL = 2u,  // rho <= 0 or p <= 0 where c is needed
  FLAG_NONFINITE = 4u,    // NaN / Inf in the new state
  FLAG_REACH = 8u,        // convective foot more than one cell from its point
  FLAG_TIMEOUT = 16u,     // a bounded wait for the CTA's own asynchronous copies ran out
  FLAG_BOUNDS = 32u       // debug builds (AF_BOUNDS_CHECK): a checked index left its region
};

template <typename T>
struct Prim {
  T r, u, v, p;
};

template <typename T>
struct PUV {
  T p, u, v;
};

// raw pointers to the sixteen planes of a state (and the four lo planes of the
// compensated averages; null unless AF_FP32_COMP)
template <typename T>
struct Planes {
  T* avg[4];
  T* pt[3][4];  // [family V, E_v, E_h][rho, u, v, p]
  T* lo[4];
};

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// ---- gas model (Sec. 2) ---------------------------------------------------
// Storage convention: density and pressure are held as offsets from a
// per-grid reference state (rho_ref, p_ref), and the energy average as an
// offset from p_ref/(gamma-1).  In FP32 this keeps the rounding of stored
// values proportional to the flow's variations rather than to the absolute
// pressure (low-Mach flows carry p ~ 1/(gamma M^2)); in FP64 the offsets are 0.
template <typename T>
struct Gas {
  T gamma, gm1, gm1inv, g_gm1;  // gamma, gamma-1, 1/(gamma-1), gamma/(gamma-1)
  T rho_ref, p_ref;
};

// The helpers below spell out their fused multiply-adds: the library is built
// without contraction, so every copy of an expression rounds the same way (a
// value computed by two thread blocks must agree bitwise for conservation).

// conservative offsets (rho~, rho u, rho v, E~) of a stored primitive
// (rho~, u, v, p~): E~ = E - p_ref/(gamma-1) = p~/(gamma-1) + rho |u|^2 / 2
template <typename T>
__device__ __forceinline__ void cons_from_stored(const Prim<T>& w, const Gas<T>& g, T u[4]) {
  const T rho = g.rho_ref + w.r;
  u[0] = w.r;
  u[1] = rho * w.u;
  u[2] = rho * w.v;
  u[3] = fma(w.p, g.gm1inv, (T(0.5) * rho) * fma(w.u, w.u, w.v * w.v));
}

// primitive from conservative offsets given 1/rho
template <typename T>
__device__ __forceinline__ Prim<T> stored_from_cons_inv(const T u[4], const Gas<T>& g, T inv) {
  Prim<T> w;
  w.r = u[0];
  w.u = u[1] * inv;
  w.v = u[2] * inv;
  w.p = g.gm1 * fma(T(-0.5), fma(u[1], w.u, u[2] * w.v), u[3]);
  return w;
}

template <typename T>
__device__ __forceinline__ Prim<T> stored_from_cons(const T u[4], const Gas<T>& g) {
  return stored_from_cons_inv(u, g, T(1) / (g.rho_ref + u[0]));
}

// Euler fluxes F (x) and G (y) of a stored primitive.  The constant p_ref is
// left out of the momentum fluxes: it cancels in every flux difference.
template <typename T>
__device__ __forceinline__ void flux_x(const Prim<T>& w, const Gas<T>& g, T f[4]) {
  const T rho = g.rho_ref + w.r, p = g.p_ref + w.p;
  const T m = rho * w.u;
  f[0] = m;
  f[1] = fma(m, w.u, w.p);
  f[2] = m * w.v;
  f[3] = w.u * fma(p, g.g_gm1, (T(0.5) * rho) * fma(w.u, w.u, w.v * w.v));
}

template <typename T>
__device__ __forceinline__ void flux_y(const Prim<T>& w, const Gas<T>& g, T f[4]) {
  const T rho = g.rho_ref + w.r, p = g.p_ref + w.p;
  const T m = rho * w.v;
  f[0] = m;
  f[1] = m * w.u;
  f[2] = fma(m, w.v, w.p);
  f[3] = w.v * fma(p, g.g_gm1, (T(0.5) * rho) * fma(w.u, w.u, w.v * w.v));
}

// ---- Q2 Lagrange basis on nodes -1, 0, 1 (Sec. 4) ----------------------------
template <typename T>
__device__ __forceinline__ void lagrange3(T s, T l[3]) {
  T hs = T(0.5) * s;
  l[0] = hs * (s - T(1));
  l[1] = T(1) - s * s;
  l[2] = hs * (s + T(1));
}

// ---- half-cell lattice ------------------------------------------------------
// Every point of the Q2 reconstruction lives on the lattice of half cells:
// lattice (I, J) = (2i + a, 2j + b) is, for (a, b) = (0,0) the vertex V(i,j),
// (0,1) the x-edge midpoint E_v(i,j), (1,0) the y-edge midpoint E_h(i,j) and
// (1,1) the centre of C_ij.  Cell C_ij owns lattice nodes 2i..2i+2 x 2j..2j+2.
__device__ __forceinline__ int lattice_family(int I, int J) {
  return (I & 1) ? ((J & 1) ? 3 : 2) : ((J & 1) ? 1 : 0);
}

// Global-memory view of the lattice: the point planes of one state plus the
// recovered centres (family 3).
template <typename T>
struct LatticeG {
  const T* f[4][4];  // [family][rho, u, v, p]
  int nx, ny;
  __device__ __forceinline__ Prim<T> at(int I, int J) const {
    int fam = lattice_family(I, J);
    int i = wrapi(I >> 1, nx), j = wrapi(J >> 1, ny);
    size_t id = (size_t)j * nx + i;
    Prim<T> w;
    w.r = f[fam][0][id];
    w.u = f[fam][1][id];
    w.v = f[fam][2][id];
    w.p = f[fam][3][id];
    return w;
  }
};

// Global-memory view of lattice increments (du, dv, dp) per family.
template <typename T>
struct IncrG {
  const T* f[4][3];
  int nx, ny;
  __device__ __forceinline__ void at(int I, int J, T d[3]) const {
    int fam = lattice_family(I, J);
    int i = wrapi(I >> 1, nx), j = wrapi(J >> 1, ny);
    size_t id = (size_t)j * nx + i;
    d[0] = f[fam][0][id];
    d[1] = f[fam][1][id];
    d[2] = f[fam][2][id];
  }
};

// ---- error-free transformations (compensated averages) ---------------------
// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Compensated average update: (hi, lo) <- (hi, lo) + (fl - fr) + (gb - gt),
// with fl, fr, gb, gt the scaled edge terms shared with the neighbouring cells.
// Every step before the last is error free (Knuth TwoSum), so each edge value
// enters its two cells with opposite signs exactly and the only rounding is
// that of the new lo word.
__device__ __forceinline__ void comp_update(float& hi, float& lo, float fl, float fr, float gb,
                                            float gt) {
  float dx, ex, dy, ey, d, ed, s, es, t, et;
  two_sum(fl, -fr, dx, ex);
  two_sum(gb, -gt, dy, ey);
  two_sum(dx, dy, d, ed);
  two_sum(hi, d, s, es);
  two_sum(lo, es, t, et);
  t = __fadd_rn(t, __fadd_rn(et, __fadd_rn(ed, __fadd_rn(ex, ey))));
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

}  // namespace af
