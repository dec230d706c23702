// af_noalloc.cu -- af_step_noalloc: one FP64 step with no allocation at all.
//
// Some callers cannot let a library allocate device memory: code that runs
// under a fixed, pre-reserved device-memory budget, or inside a host runtime
// that owns every allocation on the device and forbids stray cudaMalloc calls.
// For them this entry point runs the FP64 multi-kernel step on buffers the
// caller provides, and keeps its intermediate values (recovered centres,
// acoustic increments, half-step point values, edge fluxes, error word) in one
// fixed work area compiled into this library: a file-scope __device__ array
// that every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/af.h"
#include "af_ref_kernels.cuh"
#include "af_state_util.h"

using namespace af;

namespace {

constexpr size_t kMaxCells = AF_NOALLOC_MAX_CELLS;
// planes: centres 4, increments 2 x 4 x 3, half-step points 3 x 4, fluxes 4 + 4
constexpr size_t kPlanes = 4 + 24 + 12 + 8;
constexpr size_t kFlagsOffset = kPlanes * kMaxCells;  // in doubles, 256-byte aligned
constexpr size_t kWords = kFlagsOffset + 32;

// The work area.  In host code this name is only a stand-in for the device
// symbol; kernels receive the device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_work[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_work_ptr[kMaxDevices] = {nullptr};

// Once per device, with that device current: the device address of the work area.
af_status work_area(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AF_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_work_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_work) != cudaSuccess || !p) return AF_ERR_CUDA;
    g_work_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_work_ptr[dev];
  return AF_OK;
}

af_status status_of(unsigned f) {
  if (f & FLAG_NONPHYSICAL) return AF_ERR_NONPHYSICAL;
  if (f & FLAG_NONFINITE) return AF_ERR_NONFINITE;
  if (f & (FLAG_CFL | FLAG_REACH)) return AF_ERR_CFL;
  return AF_OK;
}

void set_planes(const af_state_f64* s, Planes<double>& p) {
  for (int k = 0; k < 4; ++k) {
    p.avg[k] = s->avg[k];
    p.pt[0][k] = s->vtx[k];
    p.pt[1][k] = s->ev[k];
    p.pt[2][k] = s->eh[k];
    p.lo[k] = nullptr;
  }
}

bool planes_ok(const af_state_f64* s) {
  if (!s) return false;
  for (int k = 0; k < 4; ++k)
    if (!s->avg[k] || !s->vtx[k] || !s->ev[k] || !s->eh[k]) return false;
  return true;
}

}  // namespace

extern "C" af_status af_step_noalloc(const af_grid* g, double gamma, double dt, af_variant var,
                                     const af_state_f64* in, const af_state_f64* out,
                                     void* cuda_stream) {
  if (!g || g->nx < 2 || g->ny < 2 || !(g->h > 0.0) || !(gamma > 1.0) || !(dt > 0.0))
    return AF_ERR_ARG;
  if ((size_t)g->nx * (size_t)g->ny > kMaxCells) return AF_ERR_ARG;  // beyond the work area
  if (var != AF_TAI && var != AF_RB) return AF_ERR_ARG;
  if (!planes_ok(in) || !planes_ok(out)) return AF_ERR_ARG;
  // the kernels write `out` while later ones still read `in`
  if (state_planes_overlap(in, out, sizeof(double) * (size_t)g->nx * (size_t)g->ny))
    return AF_ERR_ARG;
  double* work = nullptr;
  af_status st = work_area(&work);
  if (st != AF_OK) return st;

  const size_t N = (size_t)g->nx * g->ny;
  StepArgs<double> a;
  set_planes(in, a.in);
  set_planes(out, a.out);
  double* p = work;
  for (int k = 0; k < 4; ++k) a.wc[k] = p + (size_t)(0 + k) * N;
  p += 4 * N;
  for (int s = 0; s < 2; ++s)
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < 3; ++k) {
        a.inc[s][f][k] = p;
        p += N;
      }
  for (int f = 0; f < 3; ++f)
    for (int k = 0; k < 4; ++k) {
      a.half[f][k] = p;
      p += N;
    }
  for (int k = 0; k < 4; ++k) {
    a.fx[k] = p;
    p += N;
  }
  for (int k = 0; k < 4; ++k) {
    a.gy[k] = p;
    p += N;
  }
  a.flags = reinterpret_cast<unsigned*>(work + kFlagsOffset);
  a.nx = g->nx;
  a.ny = g->ny;
  a.h = g->h;
  a.dt = dt;
  a.gas.gamma = gamma;
  a.gas.gm1 = gamma - 1.0;
  a.gas.gm1inv = 1.0 / (gamma - 1.0);
  a.gas.g_gm1 = gamma / (gamma - 1.0);
  a.gas.rho_ref = 0.0;
  a.gas.p_ref = 0.0;
  a.variant = (int)var;
  a.prefetch_wave = 0;
  a.late_first_wait = 0;

  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the work area keeps the previous call's contents: the error word must start at 0
  if (cudaMemsetAsync(a.flags, 0, sizeof(unsigned), s) != cudaSuccess) return AF_ERR_CUDA;
  dim3 blk(32, 8), grd((g->nx + 31) / 32, (g->ny + 7) / 8);
  k_center<double, false><<<grd, blk, 0, s>>>(a);
  k_acoustic<0, double><<<grd, blk, 0, s>>>(a);
  k_acoustic<1, double><<<grd, blk, 0, s>>>(a);
  k_acoustic<2, double><<<grd, blk, 0, s>>>(a);
  k_acoustic<3, double><<<grd, blk, 0, s>>>(a);
  k_points<0, double><<<grd, blk, 0, s>>>(a);
  k_points<1, double><<<grd, blk, 0, s>>>(a);
  k_points<2, double><<<grd, blk, 0, s>>>(a);
  k_flux<double><<<grd, blk, 0, s>>>(a);
  k_average<double, false><<<grd, blk, 0, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return AF_ERR_CUDA;
  unsigned flags = 0;
  if (cudaMemcpyAsync(&flags, a.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return AF_ERR_CUDA;
  return status_of(flags);
}
