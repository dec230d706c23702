// af_reduce.cuh -- FP64 global diagnostics of a state: conserved totals
// (Sec. 3.1), the entropy functional -int rho log(p/rho^gamma) dA (Sec. 6),
// kinetic energy, wave-speed / positivity extrema and the vorticity integral
// (Sec. 6.4).  Two passes: per-block partials with warp shuffles, then one
// block folds the partials in a fixed order (bitwise reproducible).
#pragma once

#include "af_common.cuh"

namespace af {

enum { RED_SUMS = 8, RED_VALS = 11, RED_THREADS = 256 };
// partial layout: sums mass, mx, my, E, entropy(Simpson), entropy(avg), KE, vorticity;
// then max(|u|+c), min rho, min p

template <typename T>
struct RedArgs {
  Planes<T> st;
  const T* wc[4];
  int nx, ny;
  double gamma, h;
  double rho_ref, p_ref, e_ref;  // storage offsets (see Gas)
  double* partial;  // [gridDim.x][RED_VALS]
};

__device__ __forceinline__ double entropy_density(double r, double p, double gamma) {
  return -r * (log(p) - gamma * log(r));
}

template <typename T, bool COMP>
__global__ void __launch_bounds__(RED_THREADS) k_inv_partial(RedArgs<T> a) {
  double acc[RED_VALS];
  for (int k = 0; k < RED_SUMS; ++k) acc[k] = 0.0;
  acc[8] = 0.0;
  acc[9] = INFINITY;
  acc[10] = INFINITY;
  const size_t N = (size_t)a.nx * a.ny;
  const double sw[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
  for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < N;
       id += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(id % a.nx), j = (int)(id / a.nx);
    int ip = wrapi(i + 1, a.nx), jp = wrapi(j + 1, a.ny);
    double ub[4];
    for (int k = 0; k < 4; ++k) {
      ub[k] = (double)a.st.avg[k][id] + (COMP ? (double)a.st.lo[k][id] : 0.0);
      ub[k] += k == 0 ? a.rho_ref : (k == 3 ? a.e_ref : 0.0);
      acc[k] += ub[k];
    }
    double ra = ub[0], ua = ub[1] / ra, va = ub[2] / ra;
    double pa = (a.gamma - 1.0) * (ub[3] - 0.5 * ra * (ua * ua + va * va));
    acc[5] += entropy_density(ra, pa, a.gamma);
    acc[6] += 0.5 * (ub[1] * ub[1] + ub[2] * ub[2]) / ra;
    // The Simpson entropy integral sums, over the cells, the nine nodes of each
    // with weights (1/6, 4/6, 1/6) x (1/6, 4/6, 1/6).  On the periodic grid every
    // vertex lies in four cells, every edge midpoint in two and every centre in
    // one, so the same total is each cell's own four nodes (vertex (i, j), edges
    // (i, j+1/2) and (i+1/2, j), centre) with weights 1/9, 2/9, 2/9, 4/9: one
    // entropy evaluation (two FP64 logarithms) per node instead of per
    // cell-node pair.
    auto ld = [&](const T* const* pl, size_t q, double* o) {
      for (int k = 0; k < 4; ++k) o[k] = (double)pl[k][q];
      o[0] += a.rho_ref;
      o[3] += a.p_ref;
    };
    double wv[4], wev[4], weh[4], wcn[4];
    ld(a.st.pt[0], id, wv);
    ld(a.st.pt[1], id, wev);
    ld(a.st.pt[2], id, weh);
    ld(a.wc, id, wcn);
    acc[4] += (entropy_density(wv[0], wv[3], a.gamma) +
               2.0 * (entropy_density(wev[0], wev[3], a.gamma) +
                      entropy_density(weh[0], weh[3], a.gamma)) +
               4.0 * entropy_density(wcn[0], wcn[3], a.gamma)) /
              9.0;
    const double* own[4] = {wv, weh, wev, wcn};
    for (int n = 0; n < 4; ++n) {
      const double* o = own[n];
      double s = sqrt(o[1] * o[1] + o[2] * o[2]) + sqrt(a.gamma * o[3] / o[0]);
      acc[8] = fmax(acc[8], s);
      acc[9] = fmin(acc[9], o[0]);
      acc[10] = fmin(acc[10], o[3]);
    }
    // circulation around the cell: Simpson along its four edges (the right and
    // top edges' nodes belong to the neighbouring cells)
    const size_t q10 = (size_t)j * a.nx + ip, q01 = (size_t)jp * a.nx + i,
                 q11 = (size_t)jp * a.nx + ip;
    const double v10 = (double)a.st.pt[0][2][q10], u10 = (double)a.st.pt[0][1][q10];
    const double v11 = (double)a.st.pt[0][2][q11], u11 = (double)a.st.pt[0][1][q11];
    const double v01 = (double)a.st.pt[0][2][q01], u01 = (double)a.st.pt[0][1][q01];
    const double vev10 = (double)a.st.pt[1][2][q10], ueh01 = (double)a.st.pt[2][1][q01];
    const double vr = sw[0] * v10 + sw[1] * vev10 + sw[2] * v11;
    const double vl = sw[0] * wv[2] + sw[1] * wev[2] + sw[2] * v01;
    const double ut = sw[0] * u01 + sw[1] * ueh01 + sw[2] * u11;
    const double ubt = sw[0] * wv[1] + sw[1] * weh[1] + sw[2] * u10;
    acc[7] += a.h * (vr - vl) - a.h * (ut - ubt);
  }
  // block reduction: warp shuffles, then one warp over the warp results
  __shared__ double sh[RED_THREADS / 32][RED_VALS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < RED_VALS; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) {
      double t = __shfl_down_sync(0xffffffffu, v, o);
      v = (k < RED_SUMS) ? v + t : (k == 8 ? fmax(v, t) : fmin(v, t));
    }
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < RED_VALS) {
    int k = threadIdx.x;
    double v = sh[0][k];
    for (int wi = 1; wi < RED_THREADS / 32; ++wi)
      v = (k < RED_SUMS) ? v + sh[wi][k] : (k == 8 ? fmax(v, sh[wi][k]) : fmin(v, sh[wi][k]));
    a.partial[(size_t)blockIdx.x * RED_VALS + k] = v;
  }
}

// one block of RED_VALS threads folds nblocks partials in index order
__global__ void k_inv_final(const double* partial, int nblocks, double h, double* out) {
  int k = threadIdx.x;
  if (k >= RED_VALS) return;
  double v = partial[k];
  for (int b = 1; b < nblocks; ++b) {
    double t = partial[(size_t)b * RED_VALS + k];
    v = (k < RED_SUMS) ? v + t : (k == 8 ? fmax(v, t) : fmin(v, t));
  }
  double h2 = h * h;
  // output order follows AF_INV_*: mass, mx, my, E, entropy, entropy_avg, KE,
  // max speed, min rho, min p, vorticity
  if (k < 7) out[k] = h2 * v;
  else if (k == 7) out[10] = v;
  else out[k - 1] = v;
}

}  // namespace af
