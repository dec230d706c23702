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
  FLAG_REACH = 8u         // convective foot more than one cell from its point
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
template <typename T>
__device__ __forceinline__ void cons_from_prim(const Prim<T>& w, T gm1inv, T u[4]) {
  u[0] = w.r;
  u[1] = w.r * w.u;
  u[2] = w.r * w.v;
  u[3] = w.p * gm1inv + T(0.5) * w.r * (w.u * w.u + w.v * w.v);
}

template <typename T>
__device__ __forceinline__ Prim<T> prim_from_cons(const T u[4], T gm1) {
  Prim<T> w;
  w.r = u[0];
  T inv = T(1) / u[0];
  w.u = u[1] * inv;
  w.v = u[2] * inv;
  w.p = gm1 * (u[3] - T(0.5) * (u[1] * w.u + u[2] * w.v));
  return w;
}

// Euler fluxes F (x) and G (y) from a primitive state
template <typename T>
__device__ __forceinline__ void flux_x(const Prim<T>& w, T gm1inv, T f[4]) {
  T e = w.p * gm1inv + T(0.5) * w.r * (w.u * w.u + w.v * w.v);
  T m = w.r * w.u;
  f[0] = m;
  f[1] = m * w.u + w.p;
  f[2] = m * w.v;
  f[3] = w.u * (e + w.p);
}

template <typename T>
__device__ __forceinline__ void flux_y(const Prim<T>& w, T gm1inv, T g[4]) {
  T e = w.p * gm1inv + T(0.5) * w.r * (w.u * w.u + w.v * w.v);
  T m = w.r * w.v;
  g[0] = m;
  g[1] = m * w.u;
  g[2] = m * w.v + w.p;
  g[3] = w.v * (e + w.p);
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

}  // namespace af
