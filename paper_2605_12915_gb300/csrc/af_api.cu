// af_api.cu -- C ABI of the RB-TAI Active Flux step on GB300 (include/af.h).
// One handle = one grid on one device and one stream; the state lives in HBM as
// structure-of-arrays planes (sixteen per state, four more lo planes for the
// compensated averages), ping-ponged between steps.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <new>
#include <type_traits>

#include "../../include/af.h"
#include "af_common.cuh"
#include "af_reduce.cuh"
#include "af_ref_kernels.cuh"
#include "af_fused.cuh"
#include "af_launch.cuh"
#include "af_adjoint.cuh"
#include "af_state_util.h"

using namespace af;

namespace af {
// foot-centred point update of the three point families (af_fc.cu)
cudaError_t launch_fc_points(const StepArgs<double>& a, dim3 grd, dim3 blk, cudaStream_t s);
}  // namespace af

struct af_handle {
  int device;
  int nx, ny;
  size_t N;
  double h, gamma;
  double rho_ref, p_ref;  // storage offsets of density and pressure (0 in FP64)
  af_precision prec;
  af_variant var;
  cudaStream_t stream;
  size_t esize;          // bytes per element (4 or 8)
  void* arena;           // all device planes of this handle
  void* state[2][20];    // ping-pong state planes: 16 (+4 lo)
  int cur;               // index of the current state
  void* scratch[48];     // wc 4, inc 24, half 12, fx 4, gy 4
  double* staging;       // 16 FP64 planes for host/device exchange (lazy)
  unsigned* d_flags;
  unsigned* h_flags;     // pinned mirror, written asynchronously after each step
  unsigned* h_flags_dev; // the device's address of that mirror
  double* d_red;         // reduction partials + result
  double* h_red;         // pinned
  int red_blocks;
  int broken;
  int fused;             // 1: fused single-pass kernel for the FP32 modes
  int prefetch_wave;     // resident CTAs of the fused kernel (one wave)
  int pipe_ctas;         // CTAs of the persistent pipelined fused kernel (0: off)
  TileMaps* tmaps;       // tensor maps of the input planes of state[0], state[1]
  int tma;               // 1: the pipelined kernel stages interior tiles by tensor copies
  int zero_copy;         // 1: pinned host planes are converted in place (AF_ZERO_COPY=0: copies)
  void* adj_arena;       // adjoint arena (lazy): LAM_PLANES planes, see AdjView
  int adj_clean;         // 1: its node and increment records are zero (left so by
                         // the consumers of the last completed adjoint step)
  double* xstaging;      // 16 FP64 planes of af_exchange_state's outgoing state (lazy)
  cudaStream_t aux;      // af_exchange_state: outgoing copies (lazy)
  cudaStream_t aux_in;   // af_exchange_state: incoming copies (lazy)
  cudaEvent_t ev_fork, ev_join, ev_in;
  int late_once;         // testing only (AF_TEST_LATE_WAIT=1 at af_init): the first
                         // pipelined step reports its first staged-tile wait as timed out
  int out_pending;       // 1: the outgoing copies of the last exchange may be in flight
  af_state_f64 pending_out;  // ... into these planes
  // af_exchange_state_async (lazy): two incoming and two outgoing staging
  // buffers of 16 FP64 planes, used by alternate calls
  double* astage[2];
  double* axstage[2];
  cudaEvent_t ev_staged[2];    // the incoming copy into astage[b] is done
  cudaEvent_t ev_imported[2];  // the import that read astage[b] is done (astage[b] free)
  cudaEvent_t ev_exported[2];  // the export into axstage[b] is done
  cudaEvent_t ev_sent[2];      // the outgoing copy from axstage[b] is done (axstage[b] free)
  int abuf;                    // buffer of the next asynchronous exchange
  int apending[2];             // 1: the outgoing copy of buffer b may be in flight ...
  af_state_f64 apending_out[2];  // ... into these planes
};

namespace {

// Named NVTX range over one ABI call (profilers and timeline tools show the
// calls around the kernels they launch; without a tool attached it costs a
// pointer check).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Copies the device error word into the host's pinned mirror by a store
// through the device's mapping of page-locked memory.  No copy engine takes
// part, so the copy never waits behind large host-bound copies in flight on
// the exchange streams (a cudaMemcpyAsync of the word can queue behind them
// and hold up the step stream for a whole state transfer).
__global__ void k_flags_to_host(const unsigned* d, unsigned* h) {
  if (threadIdx.x == 0) {
    *(volatile unsigned*)h = *(volatile const unsigned*)d;
    __threadfence_system();
  }
}

af_status map_flags(unsigned f) {
  if (f & FLAG_BOUNDS) return AF_ERR_BOUNDS;
  if (f & FLAG_TIMEOUT) return AF_ERR_TIMEOUT;
  if (f & FLAG_NONPHYSICAL) return AF_ERR_NONPHYSICAL;
  if (f & FLAG_NONFINITE) return AF_ERR_NONFINITE;
  if (f & (FLAG_CFL | FLAG_REACH)) return AF_ERR_CFL;
  return AF_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <typename T>
Planes<T> planes_of(af_handle* h, int which) {
  Planes<T> p;
  void** s = h->state[which];
  for (int k = 0; k < 4; ++k) p.avg[k] = (T*)s[k];
  for (int f = 0; f < 3; ++f)
    for (int k = 0; k < 4; ++k) p.pt[f][k] = (T*)s[4 + 4 * f + k];
  for (int k = 0; k < 4; ++k) p.lo[k] = (T*)s[16 + k];
  return p;
}

// ---- FP64 <-> working precision conversion ---------------------------------
struct F64Planes {
  const double* p[16];
};
struct F64Out {
  double* p[16];
};

struct Offsets {
  double rho, p, e;  // subtracted from rho, p and the energy average on import
};

template <typename T, bool COMP>
__global__ void k_import(F64Planes src, Planes<T> dst, size_t N, Offsets o) {
  for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < N;
       id += (size_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < 4; ++k) {
      double x = src.p[k][id] - (k == 0 ? o.rho : (k == 3 ? o.e : 0.0));
      T hi = (T)x;
      dst.avg[k][id] = hi;
      if (COMP) dst.lo[k][id] = (T)(x - (double)hi);
    }
    for (int f = 0; f < 3; ++f)
      for (int k = 0; k < 4; ++k)
        dst.pt[f][k][id] =
            (T)(src.p[4 + 4 * f + k][id] - (k == 0 ? o.rho : (k == 3 ? o.p : 0.0)));
  }
}

template <typename T, bool COMP>
__global__ void k_export(Planes<T> src, F64Out dst, size_t N, Offsets o) {
  for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < N;
       id += (size_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < 4; ++k)
      dst.p[k][id] = ((double)src.avg[k][id] + (COMP ? (double)src.lo[k][id] : 0.0)) +
                     (k == 0 ? o.rho : (k == 3 ? o.e : 0.0));
    for (int f = 0; f < 3; ++f)
      for (int k = 0; k < 4; ++k)
        dst.p[4 + 4 * f + k][id] =
            (double)src.pt[f][k][id] + (k == 0 ? o.rho : (k == 3 ? o.p : 0.0));
  }
}

template <typename A, typename B>
__global__ void k_cast(const A* src, B* dst, size_t N) {
  for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < N;
       id += (size_t)gridDim.x * blockDim.x)
    dst[id] = (B)src[id];
}

Offsets offsets_of(const af_handle* h) {
  Offsets o = {h->rho_ref, h->p_ref, h->p_ref / (h->gamma - 1.0)};
  return o;
}

int grid1d(size_t N) {
  size_t b = (N + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

template <typename T>
StepArgs<T> step_args(af_handle* h, double dt) {
  StepArgs<T> a;
  a.in = planes_of<T>(h, h->cur);
  a.out = planes_of<T>(h, 1 - h->cur);
  int s = 0;
  for (int k = 0; k < 4; ++k) a.wc[k] = (T*)h->scratch[s++];
  for (int t = 0; t < 2; ++t)
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < 3; ++k) a.inc[t][f][k] = (T*)h->scratch[s++];
  for (int f = 0; f < 3; ++f)
    for (int k = 0; k < 4; ++k) a.half[f][k] = (T*)h->scratch[s++];
  for (int k = 0; k < 4; ++k) a.fx[k] = (T*)h->scratch[s++];
  for (int k = 0; k < 4; ++k) a.gy[k] = (T*)h->scratch[s++];
  a.flags = h->d_flags;
  a.nx = h->nx;
  a.ny = h->ny;
  a.h = (T)h->h;
  a.dt = (T)dt;
  a.gas.gamma = (T)h->gamma;
  a.gas.gm1 = (T)(h->gamma - 1.0);
  a.gas.gm1inv = (T)(1.0 / (h->gamma - 1.0));
  a.gas.g_gm1 = (T)(h->gamma / (h->gamma - 1.0));
  a.gas.rho_ref = (T)h->rho_ref;
  a.gas.p_ref = (T)h->p_ref;
  a.variant = (int)h->var;
  a.prefetch_wave = h->prefetch_wave;
  a.late_first_wait = 0;
  return a;
}

template <typename T, bool COMP>
void launch_ref_step(af_handle* h, double dt) {
  StepArgs<T> a = step_args<T>(h, dt);
  dim3 blk(32, 8), grd((h->nx + 31) / 32, (h->ny + 7) / 8);
  cudaStream_t s = h->stream;
  if constexpr (std::is_same<T, double>::value) {
    if (h->var == AF_FC) {  // foot-centred: no nodal increments, points from the foot disks
      k_center<T, COMP><<<grd, blk, 0, s>>>(a);
      launch_fc_points(a, grd, blk, s);
      k_flux<T><<<grd, blk, 0, s>>>(a);
      k_average<T, COMP><<<grd, blk, 0, s>>>(a);
      return;
    }
  }
  k_center<T, COMP><<<grd, blk, 0, s>>>(a);
  k_acoustic<0, T><<<grd, blk, 0, s>>>(a);
  k_acoustic<1, T><<<grd, blk, 0, s>>>(a);
  k_acoustic<2, T><<<grd, blk, 0, s>>>(a);
  k_acoustic<3, T><<<grd, blk, 0, s>>>(a);
  k_points<0, T><<<grd, blk, 0, s>>>(a);
  k_points<1, T><<<grd, blk, 0, s>>>(a);
  k_points<2, T><<<grd, blk, 0, s>>>(a);
  k_flux<T><<<grd, blk, 0, s>>>(a);
  k_average<T, COMP><<<grd, blk, 0, s>>>(a);
}

void launch_step(af_handle* h, double dt) {
  switch (h->prec) {
    case AF_FP64: launch_ref_step<double, false>(h, dt); break;
    case AF_FP32:
    case AF_FP32_COMP:
      if (h->fused) {
        StepArgs<float> a = step_args<float>(h, dt);
        a.late_first_wait = h->late_once;  // testing only, one step
        h->late_once = 0;
        if (h->prec == AF_FP32_COMP)
          launch_fused_step<true>(h->stream, a, h->pipe_ctas > 0, h->pipe_ctas,
                                  h->tma ? &h->tmaps[h->cur] : nullptr);
        else
          launch_fused_step<false>(h->stream, a, h->pipe_ctas > 0, h->pipe_ctas,
                                   h->tma ? &h->tmaps[h->cur] : nullptr);
      } else if (h->prec == AF_FP32_COMP) {
        launch_ref_step<float, true>(h, dt);
      } else {
        launch_ref_step<float, false>(h, dt);
      }
      break;
  }
}

af_status check_state_ptrs(const af_state_f64* s) {
  if (!s) return AF_ERR_ARG;
  for (int k = 0; k < 4; ++k)
    if (!s->avg[k] || !s->vtx[k] || !s->ev[k] || !s->eh[k]) return AF_ERR_ARG;
  return AF_OK;
}

const double* plane_in(const af_state_f64* s, int p) { return state_plane(s, p); }

// true when plane p of `s` starts p * N doubles after plane 0 for every p (the
// sixteen planes of one (16, ny, nx) array)
bool planes_consecutive(const af_state_f64* s, size_t N) {
  for (int p = 1; p < 16; ++p)
    if (plane_in(s, p) != plane_in(s, 0) + (size_t)p * N) return false;
  return true;
}

// Copies the sixteen planes (N doubles each) of `src` into those of `dst` on
// stream `st`: one copy when both are consecutive, else one copy per plane.
cudaError_t copy_planes(const af_state_f64* dst, const af_state_f64* src, size_t N,
                        cudaMemcpyKind kind, cudaStream_t st) {
  if (planes_consecutive(dst, N) && planes_consecutive(src, N))
    return cudaMemcpyAsync((void*)plane_in(dst, 0), plane_in(src, 0), sizeof(double) * 16 * N,
                           kind, st);
  for (int p = 0; p < 16; ++p) {
    const cudaError_t e =
        cudaMemcpyAsync((void*)plane_in(dst, p), plane_in(src, p), sizeof(double) * N, kind, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// the sixteen consecutive planes starting at `base`, as a state descriptor
af_state_f64 planes_at(double* base, size_t N) {
  af_state_f64 s;
  for (int k = 0; k < 4; ++k) {
    s.avg[k] = base + (size_t)k * N;
    s.vtx[k] = base + (size_t)(4 + k) * N;
    s.ev[k] = base + (size_t)(8 + k) * N;
    s.eh[k] = base + (size_t)(12 + k) * N;
  }
  return s;
}

af_status ensure_staging(af_handle* h) {
  if (h->staging) return AF_OK;
  if (cudaMalloc(&h->staging, sizeof(double) * 16 * h->N) != cudaSuccess) {
    h->staging = nullptr;
    return AF_ERR_ALLOC;
  }
  return AF_OK;
}

af_status cuda_fail(af_handle* h) {
  if (h) h->broken = 1;
  return AF_ERR_CUDA;
}

// Enqueues the copy of the device error word into the host mirror (read by the
// next call without waiting).
af_status flags_to_host(af_handle* h) {
  k_flags_to_host<<<1, 32, 0, h->stream>>>(h->d_flags, h->h_flags_dev);
  return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ERR_CUDA;
}

// Address under which the current device reaches the host plane p directly:
// page-locked (pinned) host memory is mapped into the device's address space
// and the import / export kernels read or write it in place over the
// host-device link.  Null for pageable memory (only the copy engines may
// touch it, through the staging buffer) or when the handle was created with
// AF_ZERO_COPY=0.
const void* mapped_host_plane(const af_handle* h, const void* p) {
  if (!h->zero_copy) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Enqueues the conversion of `in` into the current state on the handle's
// stream (pageable host planes are first copied to the staging buffer).
af_status import_enqueue(af_handle* h, const af_state_f64* in, af_memory where) {
  F64Planes src;
  if (where == AF_HOST) {
    // pinned planes are read in place by the import kernel, pageable ones are
    // copied to the staging buffer first
    for (int p = 0; p < 16; ++p) {
      src.p[p] = (const double*)mapped_host_plane(h, plane_in(in, p));
      if (src.p[p]) continue;
      af_status st = ensure_staging(h);
      if (st != AF_OK) return st;
      if (cudaMemcpyAsync(h->staging + (size_t)p * h->N, plane_in(in, p), sizeof(double) * h->N,
                          cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return cuda_fail(h);
      src.p[p] = h->staging + (size_t)p * h->N;
    }
  } else {
    for (int p = 0; p < 16; ++p) src.p[p] = plane_in(in, p);
  }
  int g = grid1d(h->N);
  switch (h->prec) {
    case AF_FP64: k_import<double, false><<<g, 256, 0, h->stream>>>(src, planes_of<double>(h, h->cur), h->N, offsets_of(h)); break;
    case AF_FP32: k_import<float, false><<<g, 256, 0, h->stream>>>(src, planes_of<float>(h, h->cur), h->N, offsets_of(h)); break;
    case AF_FP32_COMP: k_import<float, true><<<g, 256, 0, h->stream>>>(src, planes_of<float>(h, h->cur), h->N, offsets_of(h)); break;
  }
  if (cudaGetLastError() != cudaSuccess) return cuda_fail(h);
  return AF_OK;
}

// True if `in` shares a byte with the target of an outgoing copy of an
// exchange that may still be in flight.
bool overlaps_pending_out(const af_handle* h, const af_state_f64* in) {
  const size_t bytes = sizeof(double) * h->N;
  if (h->out_pending && state_planes_overlap(&h->pending_out, in, bytes)) return true;
  for (int b = 0; b < 2; ++b)
    if (h->apending[b] && state_planes_overlap(&h->apending_out[b], in, bytes)) return true;
  return false;
}

// Orders the handle's stream after the outgoing copies of earlier exchanges
// (af_exchange_state, af_exchange_state_async), which may still be in flight
// on the aux stream (ev_join follows the latest of them).
af_status wait_outgoing(af_handle* h) {
  if ((h->out_pending || h->apending[0] || h->apending[1]) &&
      cudaStreamWaitEvent(h->stream, h->ev_join, 0) != cudaSuccess)
    return cuda_fail(h);
  return AF_OK;
}

// Clears the latched device error once the stream has passed the new state
// (and, the caller having called wait_outgoing, any outgoing copies).
af_status import_finish(af_handle* h) {
  if (cudaMemsetAsync(h->d_flags, 0, sizeof(unsigned), h->stream) != cudaSuccess) return cuda_fail(h);
  if (cudaGetLastError() != cudaSuccess) return cuda_fail(h);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h);
  *(volatile unsigned*)h->h_flags = 0;
  h->out_pending = 0;
  h->apending[0] = h->apending[1] = 0;
  return AF_OK;
}

af_status import_state(af_handle* h, const af_state_f64* in, af_memory where) {
  af_status st = import_enqueue(h, in, where);
  return st != AF_OK ? st : import_finish(h);
}

// Enqueues the conversion of the current state into the FP64 planes dst.
af_status export_enqueue(af_handle* h, const F64Out& dst) {
  int g = grid1d(h->N);
  switch (h->prec) {
    case AF_FP64: k_export<double, false><<<g, 256, 0, h->stream>>>(planes_of<double>(h, h->cur), dst, h->N, offsets_of(h)); break;
    case AF_FP32: k_export<float, false><<<g, 256, 0, h->stream>>>(planes_of<float>(h, h->cur), dst, h->N, offsets_of(h)); break;
    case AF_FP32_COMP: k_export<float, true><<<g, 256, 0, h->stream>>>(planes_of<float>(h, h->cur), dst, h->N, offsets_of(h)); break;
  }
  return cudaGetLastError() == cudaSuccess ? AF_OK : cuda_fail(h);
}


}  // namespace
extern "C" af_status af_sync(af_handle* h);
namespace {

// End of an adjoint step: every kernel ran, so the records are clear again
// (unless the stream failed).
af_status adjoint_done(af_handle* h) {
  const af_status st = af_sync(h);
  h->adj_clean = (st != AF_ERR_CUDA && st != AF_ERR_STATE) ? 1 : 0;
  return st;
}

template <typename T, bool COMP>
af_status adjoint_impl(af_handle* h, double dt, const af_state_f64* lin, const af_state_f64* lout,
                       af_memory where) {
  // every plane (state, intermediates, adjoints) has the same padded size
  const size_t plane = (h->N * sizeof(T) + 255) & ~(size_t)255;
  if (!h->adj_arena && cudaMalloc(&h->adj_arena, plane * LAM_PLANES) != cudaSuccess) {
    h->adj_arena = nullptr;
    return AF_ERR_ALLOC;
  }
  const StepArgs<T> f = step_args<T>(h, dt);
  AdjView<T> v;
  v.st = (const T*)h->state[h->cur][0];
  v.sto = (const T*)h->state[1 - h->cur][0];
  v.scr = (const T*)h->scratch[0];
  v.lam = (T*)h->adj_arena;
  v.ps = plane / sizeof(T);
  v.nx = h->nx;
  v.ny = h->ny;
  v.h = f.h;
  v.dt = f.dt;
  v.gas = f.gas;
  v.variant = f.variant;
  cudaStream_t s = h->stream;
  // lambda^{n+1} in (FP64 -> working precision, no storage offsets)
  af_status st = ensure_staging(h);
  if (st != AF_OK) return st;
  Cast16<double, T> cin;
  const af_state_f64 staged = planes_at(h->staging, h->N);
  if (where == AF_HOST &&
      copy_planes(&staged, lin, h->N, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cuda_fail(h);
  for (int p = 0; p < 16; ++p) {
    const double* src = where == AF_HOST ? plane_in(&staged, p) : plane_in(lin, p);
    cin.src[p] = src;
    cin.dst[p] = v.lam + (size_t)(LAM_IN + p) * v.ps;
    v.lin64[p] = src;
  }
  dim3 blk(32, 8), grd((h->nx + 31) / 32, (h->ny + 7) / 8);
  // FP32 modes on grids the pipelined kernel accepts: one fused launch
  // recomputes each tile's step in shared memory and reverses its fluxes and
  // point updates there (AF_ADJ_FUSED=0 selects the kernel-per-stage sweep)
  if constexpr (std::is_same<T, float>::value) {
    const char* fz = getenv("AF_ADJ_FUSED");
    if (h->fused && h->pipe_ctas > 0 && pipe_eligible(f) && !(fz && fz[0] == '0')) {
      // node and increment records start at zero (planes LAM_NODE ... LAM_INC + 31):
      // cleared here only after an incomplete step or on first use, since
      // their consumers clear them as they read them
      if (!h->adj_clean &&
          cudaMemsetAsync(v.lam + (size_t)LAM_NODE * v.ps, 0, plane * 48, s) != cudaSuccess)
        return cuda_fail(h);
      h->adj_clean = 0;
      if (launch_fused_adjoint<COMP>(s, f, h->pipe_ctas, h->tma ? &h->tmaps[h->cur] : nullptr,
                                     v) != cudaSuccess)
        return cuda_fail(h);
      k_adj_acoustic<0, T><<<grd, blk, 0, s>>>(v);
      k_adj_acoustic<1, T><<<grd, blk, 0, s>>>(v);
      k_adj_acoustic<2, T><<<grd, blk, 0, s>>>(v);
      k_adj_acoustic<3, T><<<grd, blk, 0, s>>>(v);
      k_adj_center<T><<<grd, blk, 0, s>>>(v);
      AdjOut<T> out;
      for (int p = 0; p < 16; ++p)
        out.dst[p] = where == AF_HOST ? h->staging + (size_t)p * h->N : (double*)plane_in(lout, p);
      k_adj_out<T><<<grid1d(h->N), 256, 0, s>>>(v, out, h->N);
      if (where == AF_HOST &&
          copy_planes(lout, &staged, h->N, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return cuda_fail(h);
      if (cudaGetLastError() != cudaSuccess) return cuda_fail(h);
      return adjoint_done(h);
    }
  }
  // the stage-by-stage sweep reads lambda^{n+1} in the working precision
  k_cast16<<<grid1d(h->N), 256, 0, s>>>(cin, h->N);
  // forward intermediates of the step from the handle's current state: the
  // pipelined fused kernel stores them where it runs (FP32 modes), else the
  // unfused kernels
  bool fused_inter = false;
  if constexpr (std::is_same<T, float>::value) {
    if (h->fused && h->pipe_ctas > 0 && pipe_eligible(f)) {
      if (launch_fused_step<COMP, true>(s, f, true, h->pipe_ctas,
                                        h->tma ? &h->tmaps[h->cur] : nullptr) != cudaSuccess)
        return cuda_fail(h);
      fused_inter = true;
    }
  }
  if (!fused_inter) {
    k_center<T, COMP><<<grd, blk, 0, s>>>(f);
    k_acoustic<0, T><<<grd, blk, 0, s>>>(f);
    k_acoustic<1, T><<<grd, blk, 0, s>>>(f);
    k_acoustic<2, T><<<grd, blk, 0, s>>>(f);
    k_acoustic<3, T><<<grd, blk, 0, s>>>(f);
    k_points<0, T><<<grd, blk, 0, s>>>(f);
    k_points<1, T><<<grd, blk, 0, s>>>(f);
    k_points<2, T><<<grd, blk, 0, s>>>(f);
  }
  // reverse sweep: the centre and increment records start at zero (planes
  // LAM_NODE + 12 ... LAM_INC + 31 are contiguous; the sweep writes the other
  // node records before adding to them)
  if (!h->adj_clean &&
      cudaMemsetAsync(v.lam + (size_t)(LAM_NODE + 12) * v.ps, 0, plane * 36, s) != cudaSuccess)
    return cuda_fail(h);
  h->adj_clean = 0;
  k_adj_flux<T><<<grd, blk, 0, s>>>(v);
  k_adj_points<0, T><<<grd, blk, 0, s>>>(v);
  k_adj_points<1, T><<<grd, blk, 0, s>>>(v);
  k_adj_points<2, T><<<grd, blk, 0, s>>>(v);
  k_adj_acoustic<0, T><<<grd, blk, 0, s>>>(v);
  k_adj_acoustic<1, T><<<grd, blk, 0, s>>>(v);
  k_adj_acoustic<2, T><<<grd, blk, 0, s>>>(v);
  k_adj_acoustic<3, T><<<grd, blk, 0, s>>>(v);
  k_adj_center<T><<<grd, blk, 0, s>>>(v);
  // lambda^n out
  AdjOut<T> out;
  for (int p = 0; p < 16; ++p)
    out.dst[p] = where == AF_HOST ? h->staging + (size_t)p * h->N : (double*)plane_in(lout, p);
  k_adj_out<T><<<grid1d(h->N), 256, 0, s>>>(v, out, h->N);
  if (where == AF_HOST &&
      copy_planes(lout, &staged, h->N, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cuda_fail(h);
  if (cudaGetLastError() != cudaSuccess) return cuda_fail(h);
  return adjoint_done(h);
}

}  // namespace

extern "C" {

const char* af_status_string(af_status s) {
  switch (s) {
    case AF_OK: return "ok";
    case AF_ERR_ARG: return "invalid argument";
    case AF_ERR_CUDA: return "CUDA runtime error";
    case AF_ERR_ALLOC: return "allocation failed";
    case AF_ERR_CFL: return "time step too large: acoustic CFL above 1/2 or convective foot beyond one cell";
    case AF_ERR_NONPHYSICAL: return "non-positive density or pressure";
    case AF_ERR_NONFINITE: return "non-finite value in the state";
    case AF_ERR_STATE: return "handle unusable after a CUDA error";
    case AF_ERR_TIMEOUT: return "a device-side wait for asynchronous copies timed out";
    case AF_ERR_BOUNDS: return "a checked kernel index left its region (bounds-checking build)";
  }
  return "unknown status";
}

af_status af_init(af_handle** out, const af_grid* g, double gamma, const af_state_f64* state,
                  af_memory where, af_precision prec, af_variant var, void* cuda_stream) {
  if (!out) return AF_ERR_ARG;
  *out = nullptr;
  if (!g || g->nx < 2 || g->ny < 2 || !(g->h > 0.0) || !(gamma > 1.0)) return AF_ERR_ARG;
  if (prec != AF_FP64 && prec != AF_FP32 && prec != AF_FP32_COMP) return AF_ERR_ARG;
  if (var != AF_TAI && var != AF_RB && var != AF_FC) return AF_ERR_ARG;
  if (var == AF_FC && prec != AF_FP64) return AF_ERR_ARG;  // FP64 reference variant only
  if (where != AF_HOST && where != AF_DEVICE) return AF_ERR_ARG;
  if (check_state_ptrs(state) != AF_OK) return AF_ERR_ARG;
  if ((int64_t)g->nx * (int64_t)g->ny > (int64_t)1 << 31) return AF_ERR_ARG;

  af_handle* h = new (std::nothrow) af_handle();
  if (!h) return AF_ERR_ALLOC;
  memset(h, 0, sizeof(*h));
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return AF_ERR_CUDA;
  }
  h->nx = g->nx;
  h->ny = g->ny;
  h->N = (size_t)g->nx * g->ny;
  h->h = g->h;
  h->gamma = gamma;
  h->prec = prec;
  h->var = var;
  h->stream = (cudaStream_t)cuda_stream;
  h->esize = prec == AF_FP64 ? 8 : 4;
  // FP32 modes run the fused single-pass kernel; AF_PATH=ref selects the
  // multi-kernel path (same arithmetic, intermediate values in HBM).
  const char* path = getenv("AF_PATH");
  h->fused = (prec != AF_FP64) && !(path && strcmp(path, "ref") == 0);
  {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const char* pf = getenv("AF_PREFETCH");
    h->prefetch_wave = (pf && pf[0] == '0') ? 0 : sms * AF_FUSED_MINB;
    // persistent pipelined fused kernel on one wave of CTAs; AF_PIPE=0 selects
    // the one-CTA-per-tile kernel (same arithmetic), AF_PIPE=n > 0 caps the
    // persistent grid at n CTAs
    const char* pp = getenv("AF_PIPE");
    const int cap = pp ? atoi(pp) : 0;
    h->pipe_ctas = !pp ? sms * AF_FUSED_MINB : (cap > 0 ? std::min(cap, sms * AF_FUSED_MINB) : 0);
  }
  {
    const char* zc = getenv("AF_ZERO_COPY");
    h->zero_copy = (zc && zc[0] == '0') ? 0 : 1;
    // testing the timeout path: the handle's first pipelined step gives up its
    // first wait for a tensor-copied tile at once (the copies still complete)
    const char* lw = getenv("AF_TEST_LATE_WAIT");
    h->late_once = (lw && lw[0] == '1') ? 1 : 0;
  }
  // 2 x 20 state planes + 48 scratch planes, each padded to 256 bytes
  size_t plane = (h->N * h->esize + 255) & ~(size_t)255;
  size_t nplanes = 2 * 20 + 48;
  if (cudaMalloc(&h->arena, plane * nplanes) != cudaSuccess) {
    delete h;
    return AF_ERR_ALLOC;
  }
  char* base = (char*)h->arena;
  for (int s = 0; s < 2; ++s)
    for (int p = 0; p < 20; ++p) h->state[s][p] = base + plane * (size_t)(20 * s + p);
  for (int p = 0; p < 48; ++p) h->scratch[p] = base + plane * (size_t)(40 + p);
  h->red_blocks = 152 * 4;
  bool ok = cudaMalloc(&h->d_flags, sizeof(unsigned)) == cudaSuccess &&
            cudaMallocHost(&h->h_flags, sizeof(unsigned)) == cudaSuccess &&
            cudaHostGetDevicePointer((void**)&h->h_flags_dev, h->h_flags, 0) == cudaSuccess &&
            cudaMalloc(&h->d_red, sizeof(double) * (RED_VALS * h->red_blocks + AF_NINV)) ==
                cudaSuccess &&
            cudaMallocHost(&h->h_red, sizeof(double) * AF_NINV) == cudaSuccess;
  if (!ok) {
    af_destroy(h);
    return AF_ERR_ALLOC;
  }
  if (prec != AF_FP64 && h->pipe_ctas > 0) {
    // tensor maps of both state buffers for the pipelined kernel; AF_TMA=0 (or a
    // driver without the encoder) stages every tile by cp.async instead
    const char* tv = getenv("AF_TMA");
    h->tmaps = new (std::nothrow) TileMaps[2];
    bool enc = h->tmaps && !(tv && tv[0] == '0');
    for (int b = 0; b < 2 && enc; ++b) {
      StepArgs<float> a = {};
      a.in = planes_of<float>(h, b);
      a.nx = h->nx;
      a.ny = h->ny;
      enc = pipe_eligible(a) && encode_tile_maps(a, &h->tmaps[b]);
    }
    h->tma = enc ? 1 : 0;
  }
  if (prec == AF_FP32_COMP || prec == AF_FP32) {
    // zero the lo planes once (unused in AF_FP32)
    for (int s = 0; s < 2; ++s)
      for (int k = 16; k < 20; ++k) cudaMemsetAsync(h->state[s][k], 0, plane, h->stream);
  }
  // storage offsets: the initial vertex state at (0,0) (FP32 modes only)
  if (prec != AF_FP64) {
    double r0 = 0.0, p0 = 0.0;
    if (where == AF_HOST) {
      r0 = state->vtx[0][0];
      p0 = state->vtx[3][0];
    } else if (cudaMemcpy(&r0, state->vtx[0], sizeof(double), cudaMemcpyDeviceToHost) !=
                   cudaSuccess ||
               cudaMemcpy(&p0, state->vtx[3], sizeof(double), cudaMemcpyDeviceToHost) !=
                   cudaSuccess) {
      af_destroy(h);
      return AF_ERR_CUDA;
    }
    h->rho_ref = (r0 > 0.0 && r0 < 1e30) ? r0 : 0.0;
    h->p_ref = (p0 > 0.0 && p0 < 1e30) ? p0 : 0.0;
  }
  af_status st = import_state(h, state, where);
  if (st != AF_OK) {
    af_destroy(h);
    return st;
  }
  *out = h;
  return AF_OK;
}

af_status af_step(af_handle* h, double dt, int32_t n_steps) {
  NvtxRange range("af_step");
  if (!h) return AF_ERR_ARG;
  if (h->broken) return AF_ERR_STATE;
  if (!(dt > 0.0) || n_steps < 0) return AF_ERR_ARG;
  af_status prior = map_flags(*(volatile unsigned*)h->h_flags);
  if (prior != AF_OK) return prior;
  DeviceGuard guard(h->device);
  for (int n = 0; n < n_steps; ++n) {
    launch_step(h, dt);
    h->cur = 1 - h->cur;
  }
  if (cudaGetLastError() != cudaSuccess) return cuda_fail(h);
  if (flags_to_host(h) != AF_OK) return cuda_fail(h);
  return AF_OK;
}

af_status af_sync(af_handle* h) {
  if (!h) return AF_ERR_ARG;
  if (h->broken) return AF_ERR_STATE;
  DeviceGuard guard(h->device);
  if (wait_outgoing(h) != AF_OK) return AF_ERR_CUDA;
  if (flags_to_host(h) != AF_OK || cudaStreamSynchronize(h->stream) != cudaSuccess)
    return cuda_fail(h);
  h->out_pending = 0;
  h->apending[0] = h->apending[1] = 0;
  return map_flags(*(volatile unsigned*)h->h_flags);
}

af_status af_set_state(af_handle* h, const af_state_f64* in, af_memory where) {
  if (!h || check_state_ptrs(in) != AF_OK || (where != AF_HOST && where != AF_DEVICE))
    return AF_ERR_ARG;
  if (h->broken) return AF_ERR_STATE;
  DeviceGuard guard(h->device);
  if (wait_outgoing(h) != AF_OK) return AF_ERR_CUDA;
  return import_state(h, in, where);
}

af_status af_get_state(af_handle* h, const af_state_f64* out, af_memory where) {
  if (!h || check_state_ptrs(out) != AF_OK || (where != AF_HOST && where != AF_DEVICE))
    return AF_ERR_ARG;
  if (h->broken) return AF_ERR_STATE;
  DeviceGuard guard(h->device);
  if (wait_outgoing(h) != AF_OK) return AF_ERR_CUDA;
  F64Out dst;
  bool copy_back[16] = {};
  if (where == AF_HOST) {
    // pinned planes are written in place by the export kernel, pageable ones
    // through the staging buffer
    for (int p = 0; p < 16; ++p) {
      dst.p[p] = (double*)mapped_host_plane(h, plane_in(out, p));
      if (dst.p[p]) continue;
      af_status st = ensure_staging(h);
      if (st != AF_OK) return st;
      dst.p[p] = h->staging + (size_t)p * h->N;
      copy_back[p] = true;
    }
  } else {
    for (int p = 0; p < 16; ++p) dst.p[p] = (double*)plane_in(out, p);
  }
  af_status est = export_enqueue(h, dst);
  if (est != AF_OK) return est;
  for (int p = 0; p < 16; ++p)
    if (copy_back[p] &&
        cudaMemcpyAsync((void*)plane_in(out, p), dst.p[p], sizeof(double) * h->N,
                        cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
      return cuda_fail(h);
  return af_sync(h);
}

}  // extern "C"
namespace {

// The copy streams and events of the exchanges (created on first use).
af_status ensure_aux(af_handle* h) {
  if (h->aux) return AF_OK;
  if (cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->aux_in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess)
    return AF_ERR_CUDA;
  return AF_OK;
}

}  // namespace
extern "C" {

af_status af_exchange_state(af_handle* h, const af_state_f64* out, const af_state_f64* in,
                            af_memory where) {
  NvtxRange range("af_exchange_state");
  if (!h || check_state_ptrs(out) != AF_OK || check_state_ptrs(in) != AF_OK ||
      (where != AF_HOST && where != AF_DEVICE))
    return AF_ERR_ARG;
  if (state_planes_overlap(out, in, sizeof(double) * h->N)) return AF_ERR_ARG;
  if (h->broken) return AF_ERR_STATE;
  DeviceGuard guard(h->device);
  if (wait_outgoing(h) != AF_OK) return AF_ERR_CUDA;
  if (where == AF_DEVICE) {
    F64Out dst;
    for (int p = 0; p < 16; ++p) dst.p[p] = (double*)plane_in(out, p);
    af_status st = export_enqueue(h, dst);
    if (st == AF_OK) st = import_enqueue(h, in, AF_DEVICE);
    return st != AF_OK ? st : import_finish(h);
  }
  // host: both directions by copy engines, on two streams of their own, so that
  // they overlap on the link with each other and with the step still running:
  //   aux_in  in -> staging (FP64)                       (starts at once)
  //   stream  [earlier work] state -> xstaging (export), then, once aux_in is
  //           done, staging -> state (import)
  //   aux     xstaging -> out, after the export; left in flight on return
  if (!h->xstaging && cudaMalloc(&h->xstaging, sizeof(double) * 16 * h->N) != cudaSuccess) {
    h->xstaging = nullptr;
    return AF_ERR_ALLOC;
  }
  af_status st = ensure_staging(h);
  if (st != AF_OK) return st;
  if (ensure_aux(h) != AF_OK) return cuda_fail(h);
  // an incoming plane that is also the target of an earlier exchange's
  // outgoing copies is read after them
  if (overlaps_pending_out(h, in) && cudaStreamWaitEvent(h->aux_in, h->ev_join, 0) != cudaSuccess)
    return cuda_fail(h);
  // the staging buffer is idle: every earlier call that used it has synchronised
  const af_state_f64 staged = planes_at(h->staging, h->N);
  if (copy_planes(&staged, in, h->N, cudaMemcpyHostToDevice, h->aux_in) != cudaSuccess)
    return cuda_fail(h);
  if (cudaEventRecord(h->ev_in, h->aux_in) != cudaSuccess) return cuda_fail(h);
  F64Out dst;
  for (int p = 0; p < 16; ++p) dst.p[p] = h->xstaging + (size_t)p * h->N;
  st = export_enqueue(h, dst);
  if (st != AF_OK) return st;
  if (cudaEventRecord(h->ev_fork, h->stream) != cudaSuccess ||
      cudaStreamWaitEvent(h->aux, h->ev_fork, 0) != cudaSuccess)
    return cuda_fail(h);
  const af_state_f64 xs = planes_at(h->xstaging, h->N);
  if (copy_planes(out, &xs, h->N, cudaMemcpyDeviceToHost, h->aux) != cudaSuccess)
    return cuda_fail(h);
  if (cudaEventRecord(h->ev_join, h->aux) != cudaSuccess ||
      cudaStreamWaitEvent(h->stream, h->ev_in, 0) != cudaSuccess)
    return cuda_fail(h);
  st = import_enqueue(h, &staged, AF_DEVICE);
  if (st == AF_OK) st = import_finish(h);
  if (st == AF_OK) {
    h->out_pending = 1;
    h->pending_out = *out;
  }
  return st;
}

af_status af_exchange_state_async(af_handle* h, const af_state_f64* out,
                                  const af_state_f64* in) {
  NvtxRange range("af_exchange_state_async");
  if (!h || check_state_ptrs(out) != AF_OK || check_state_ptrs(in) != AF_OK) return AF_ERR_ARG;
  if (state_planes_overlap(out, in, sizeof(double) * h->N)) return AF_ERR_ARG;
  if (h->broken) return AF_ERR_STATE;
  DeviceGuard guard(h->device);
  if (ensure_aux(h) != AF_OK) return cuda_fail(h);
  if (!h->astage[0]) {
    const size_t bytes = sizeof(double) * 16 * h->N;
    for (int b = 0; b < 2; ++b) {
      if (cudaMalloc(&h->astage[b], bytes) != cudaSuccess) h->astage[b] = nullptr;
      if (cudaMalloc(&h->axstage[b], bytes) != cudaSuccess) h->axstage[b] = nullptr;
    }
    if (!h->astage[0] || !h->astage[1] || !h->axstage[0] || !h->axstage[1]) {
      for (int b = 0; b < 2; ++b) {
        if (h->astage[b]) cudaFree(h->astage[b]);
        if (h->axstage[b]) cudaFree(h->axstage[b]);
        h->astage[b] = h->axstage[b] = nullptr;
      }
      return AF_ERR_ALLOC;
    }
    for (int b = 0; b < 2; ++b)
      if (cudaEventCreateWithFlags(&h->ev_staged[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_imported[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_exported[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_sent[b], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(h);
  }
  const int b = h->abuf;
  const size_t N = h->N;
  const af_state_f64 staged = planes_at(h->astage[b], N);
  // incoming: into astage[b] once the import that last read it is done, and
  // after any outgoing copy still writing the planes it reads
  if (overlaps_pending_out(h, in) && cudaStreamWaitEvent(h->aux_in, h->ev_join, 0) != cudaSuccess)
    return cuda_fail(h);
  if (cudaStreamWaitEvent(h->aux_in, h->ev_imported[b], 0) != cudaSuccess) return cuda_fail(h);
  if (copy_planes(&staged, in, N, cudaMemcpyHostToDevice, h->aux_in) != cudaSuccess)
    return cuda_fail(h);
  if (cudaEventRecord(h->ev_staged[b], h->aux_in) != cudaSuccess) return cuda_fail(h);
  // outgoing: the current state into axstage[b] once its last copy out is done
  F64Out dst;
  for (int p = 0; p < 16; ++p) dst.p[p] = h->axstage[b] + (size_t)p * N;
  if (cudaStreamWaitEvent(h->stream, h->ev_sent[b], 0) != cudaSuccess) return cuda_fail(h);
  af_status st = export_enqueue(h, dst);
  if (st != AF_OK) return st;
  if (cudaEventRecord(h->ev_exported[b], h->stream) != cudaSuccess ||
      cudaStreamWaitEvent(h->aux, h->ev_exported[b], 0) != cudaSuccess)
    return cuda_fail(h);
  const af_state_f64 xs = planes_at(h->axstage[b], N);
  if (copy_planes(out, &xs, N, cudaMemcpyDeviceToHost, h->aux) != cudaSuccess)
    return cuda_fail(h);
  if (cudaEventRecord(h->ev_sent[b], h->aux) != cudaSuccess ||
      cudaEventRecord(h->ev_join, h->aux) != cudaSuccess)
    return cuda_fail(h);
  // the new state, on the handle's stream after the incoming copy
  if (cudaStreamWaitEvent(h->stream, h->ev_staged[b], 0) != cudaSuccess) return cuda_fail(h);
  st = import_enqueue(h, &staged, AF_DEVICE);
  if (st != AF_OK) return st;
  if (cudaEventRecord(h->ev_imported[b], h->stream) != cudaSuccess) return cuda_fail(h);
  h->apending[b] = 1;
  h->apending_out[b] = *out;
  h->abuf = 1 - b;
  return cudaGetLastError() == cudaSuccess ? AF_OK : cuda_fail(h);
}

af_status af_reduce_invariants(af_handle* h, double* out) {
  NvtxRange range("af_reduce_invariants");
  if (!h || !out) return AF_ERR_ARG;
  if (h->broken) return AF_ERR_STATE;
  DeviceGuard guard(h->device);
  if (wait_outgoing(h) != AF_OK) return AF_ERR_CUDA;
  double* partial = h->d_red;
  double* res = h->d_red + (size_t)RED_VALS * h->red_blocks;
  dim3 blk(32, 8), grd((h->nx + 31) / 32, (h->ny + 7) / 8);
  if (h->prec == AF_FP64) {
    StepArgs<double> a = step_args<double>(h, 1.0);
    k_center<double, false><<<grd, blk, 0, h->stream>>>(a);
    RedArgs<double> r;
    r.st = a.in;
    for (int k = 0; k < 4; ++k) r.wc[k] = a.wc[k];
    r.nx = h->nx; r.ny = h->ny; r.gamma = h->gamma; r.h = h->h; r.partial = partial;
    r.rho_ref = h->rho_ref; r.p_ref = h->p_ref; r.e_ref = h->p_ref / (h->gamma - 1.0);
    k_inv_partial<double, false><<<h->red_blocks, RED_THREADS, 0, h->stream>>>(r);
  } else {
    StepArgs<float> a = step_args<float>(h, 1.0);
    RedArgs<float> r;
    r.st = a.in;
    for (int k = 0; k < 4; ++k) r.wc[k] = a.wc[k];
    r.nx = h->nx; r.ny = h->ny; r.gamma = h->gamma; r.h = h->h; r.partial = partial;
    r.rho_ref = h->rho_ref; r.p_ref = h->p_ref; r.e_ref = h->p_ref / (h->gamma - 1.0);
    if (h->prec == AF_FP32_COMP) {
      k_center<float, true><<<grd, blk, 0, h->stream>>>(a);
      k_inv_partial<float, true><<<h->red_blocks, RED_THREADS, 0, h->stream>>>(r);
    } else {
      k_center<float, false><<<grd, blk, 0, h->stream>>>(a);
      k_inv_partial<float, false><<<h->red_blocks, RED_THREADS, 0, h->stream>>>(r);
    }
  }
  k_inv_final<<<1, 32, 0, h->stream>>>(partial, h->red_blocks, h->h, res);
  if (cudaGetLastError() != cudaSuccess) return cuda_fail(h);
  if (cudaMemcpyAsync(h->h_red, res, sizeof(double) * (AF_NINV - 1), cudaMemcpyDeviceToHost,
                      h->stream) != cudaSuccess)
    return cuda_fail(h);
  af_status st = af_sync(h);
  if (st == AF_ERR_CUDA || st == AF_ERR_STATE) return st;
  for (int k = 0; k < AF_NINV - 1; ++k) out[k] = h->h_red[k];
  out[AF_INV_FLAGS] = (double)*(volatile unsigned*)h->h_flags;
  return st;
}

af_status af_adjoint_step(af_handle* h, double dt, const af_state_f64* lam_in,
                          const af_state_f64* lam_out, af_memory where) {
  NvtxRange range("af_adjoint_step");
  if (!h || !(dt > 0.0) || check_state_ptrs(lam_in) != AF_OK ||
      check_state_ptrs(lam_out) != AF_OK || (where != AF_HOST && where != AF_DEVICE))
    return AF_ERR_ARG;
  if (h->broken) return AF_ERR_STATE;
  if (h->var == AF_FC) return AF_ERR_ARG;  // no adjoint of the foot-centred update
  DeviceGuard guard(h->device);
  if (wait_outgoing(h) != AF_OK) return AF_ERR_CUDA;
  switch (h->prec) {
    case AF_FP64: return adjoint_impl<double, false>(h, dt, lam_in, lam_out, where);
    case AF_FP32: return adjoint_impl<float, false>(h, dt, lam_in, lam_out, where);
    case AF_FP32_COMP: return adjoint_impl<float, true>(h, dt, lam_in, lam_out, where);
  }
  return AF_ERR_ARG;
}

void af_destroy(af_handle* h) {
  if (!h) return;
  DeviceGuard guard(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->aux) {  // an exchange's outgoing copy may still read xstaging
    cudaStreamSynchronize(h->aux);
    cudaStreamSynchronize(h->aux_in);
  }
  if (h->arena) cudaFree(h->arena);
  if (h->staging) cudaFree(h->staging);
  if (h->d_flags) cudaFree(h->d_flags);
  if (h->h_flags) cudaFreeHost(h->h_flags);
  if (h->d_red) cudaFree(h->d_red);
  if (h->adj_arena) cudaFree(h->adj_arena);
  if (h->xstaging) cudaFree(h->xstaging);
  if (h->astage[0]) {
    for (int b = 0; b < 2; ++b) {
      cudaFree(h->astage[b]);
      cudaFree(h->axstage[b]);
      cudaEventDestroy(h->ev_staged[b]);
      cudaEventDestroy(h->ev_imported[b]);
      cudaEventDestroy(h->ev_exported[b]);
      cudaEventDestroy(h->ev_sent[b]);
    }
  }
  if (h->aux) {
    cudaStreamDestroy(h->aux);
    cudaStreamDestroy(h->aux_in);
    cudaEventDestroy(h->ev_fork);
    cudaEventDestroy(h->ev_join);
    cudaEventDestroy(h->ev_in);
  }
  if (h->h_red) cudaFreeHost(h->h_red);
  delete[] h->tmaps;
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched ensembles: many independent grids advanced by one launch per step
// (a tile table spanning all grids), the launches of a call captured once in a
// CUDA graph; the tile geometry is chosen by timing the candidates.
// ---------------------------------------------------------------------------
struct af_batch {
  int n;
  af_handle** h;
  cudaStream_t stream;
  af_precision prec;
  StepArgs<float>* h_args;  // pinned host copy [2][n]
  StepArgs<float>* d_args;  // device [2][n]: parity p = the handles' current buffer
  int4* d_tiles[N_BATCH_GEOMS];
  int ntiles[N_BATCH_GEOMS];
  int geom;                 // -1 until tuned
  float tune_ms[N_BATCH_GEOMS];
  cudaGraphExec_t graph;
  int graph_steps, graph_parity;
  void* snapshot;           // device copy of every state while tuning
  int own_stream;           // the batch created its stream (the legacy stream cannot be captured)
  int pipe_ok;              // every grid meets the persistent kernel's staging conditions
  int pipe_ctas;            // its CTAs
  TileMaps* d_maps[2];      // device, one per grid and parity (null: cp.async staging only)
};

namespace {

af_status batch_launch(af_batch* b, int geom, int parity) {
  const StepArgs<float>* args = b->d_args + (size_t)parity * b->n;
  if (BATCH_GEOMS[geom].pipe && !b->pipe_ok) return AF_ERR_ARG;
  cudaError_t e = b->prec == AF_FP32_COMP
                      ? launch_batch<true>(geom, b->stream, args, b->d_tiles[geom], b->ntiles[geom],
                                           b->d_maps[parity], b->pipe_ctas)
                      : launch_batch<false>(geom, b->stream, args, b->d_tiles[geom],
                                            b->ntiles[geom], b->d_maps[parity], b->pipe_ctas);
  return e == cudaSuccess ? AF_OK : AF_ERR_CUDA;
}

int batch_parity(const af_batch* b) { return b->h[0]->cur; }

void batch_flip(af_batch* b, int n_steps) {
  if (n_steps & 1)
    for (int k = 0; k < b->n; ++k) b->h[k]->cur ^= 1;
}

size_t state_plane_bytes(const af_handle* h) { return (h->N * h->esize + 255) & ~(size_t)255; }

af_status batch_snapshot(af_batch* b, bool restore) {
  char* p = (char*)b->snapshot;
  for (int k = 0; k < b->n; ++k) {
    af_handle* h = b->h[k];
    const size_t bytes = state_plane_bytes(h);
    for (int q = 0; q < 20; ++q) {
      void* live = h->state[h->cur][q];
      if (cudaMemcpyAsync(restore ? live : (void*)p, restore ? (void*)p : live, bytes,
                          cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
        return AF_ERR_CUDA;
      p += bytes;
    }
  }
  return AF_OK;
}

af_status batch_tune(af_batch* b) {
  size_t total = 0;
  for (int k = 0; k < b->n; ++k) total += 20 * state_plane_bytes(b->h[k]);
  if (cudaMalloc(&b->snapshot, total) != cudaSuccess) {
    b->snapshot = nullptr;
    return AF_ERR_ALLOC;
  }
  af_status st = batch_snapshot(b, false);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int g = 0; g < N_BATCH_GEOMS && st == AF_OK; ++g) {
    b->tune_ms[g] = -1.f;
    if (BATCH_GEOMS[g].pipe && !b->pipe_ok) continue;
    int parity = batch_parity(b);
    st = batch_launch(b, g, parity);  // warm-up, attribute set-up
    parity ^= 1;
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < 2 && st == AF_OK; ++r, parity ^= 1) st = batch_launch(b, g, parity);
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    b->tune_ms[g] = ms / 2;
    if (ms < best) {
      best = ms;
      b->geom = g;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == AF_OK) st = batch_snapshot(b, true);  // three steps per candidate: parity unchanged
  for (int k = 0; k < b->n; ++k) cudaMemsetAsync(b->h[k]->d_flags, 0, sizeof(unsigned), b->stream);
  cudaStreamSynchronize(b->stream);
  cudaFree(b->snapshot);
  b->snapshot = nullptr;
  return st;
}

}  // namespace

extern "C" {

af_status af_batch_init(af_batch** out, int32_t n, const af_grid* grids, double gamma,
                        const af_state_f64* states, af_memory where, af_precision prec,
                        af_variant var, void* cuda_stream) {
  if (!out) return AF_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !grids || !states || (prec != AF_FP32 && prec != AF_FP32_COMP)) return AF_ERR_ARG;
  if (var != AF_TAI && var != AF_RB) return AF_ERR_ARG;
  af_batch* b = new (std::nothrow) af_batch();
  if (!b) return AF_ERR_ALLOC;
  memset(b, 0, sizeof(*b));
  b->n = n;
  b->prec = prec;
  b->stream = (cudaStream_t)cuda_stream;
  b->geom = -1;
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return AF_ERR_CUDA;
    }
    b->own_stream = 1;
  }
  b->h = new (std::nothrow) af_handle*[n]();
  if (!b->h) {
    delete b;
    return AF_ERR_ALLOC;
  }
  for (int k = 0; k < n; ++k) {
    af_status st = af_init(&b->h[k], &grids[k], gamma, &states[k], where, prec, var, b->stream);
    if (st != AF_OK) {
      af_batch_destroy(b);
      return st;
    }
  }
  // tile tables, largest grids first
  int* order = new int[n];
  for (int k = 0; k < n; ++k) order[k] = k;
  for (int x = 1; x < n; ++x)
    for (int y = x; y > 0 && b->h[order[y]]->N > b->h[order[y - 1]]->N; --y) {
      int t = order[y];
      order[y] = order[y - 1];
      order[y - 1] = t;
    }
  bool ok = true;
  for (int g = 0; g < N_BATCH_GEOMS && ok; ++g) {
    const int tx = BATCH_GEOMS[g].tx, ty = BATCH_GEOMS[g].ty;
    size_t cnt = 0;
    for (int k = 0; k < n; ++k)
      cnt += (size_t)((b->h[k]->nx + tx - 1) / tx) * ((b->h[k]->ny + ty - 1) / ty);
    int4* tt = new int4[cnt];
    size_t c = 0;
    for (int o = 0; o < n; ++o) {
      const int k = order[o];
      for (int j0 = 0; j0 < b->h[k]->ny; j0 += ty)
        for (int i0 = 0; i0 < b->h[k]->nx; i0 += tx) tt[c++] = make_int4(k, i0, j0, 0);
    }
    b->ntiles[g] = (int)cnt;
    ok = cudaMalloc(&b->d_tiles[g], sizeof(int4) * cnt) == cudaSuccess &&
         cudaMemcpy(b->d_tiles[g], tt, sizeof(int4) * cnt, cudaMemcpyHostToDevice) == cudaSuccess;
    delete[] tt;
  }
  delete[] order;
  ok = ok && cudaMallocHost(&b->h_args, sizeof(StepArgs<float>) * 2 * n) == cudaSuccess &&
       cudaMalloc(&b->d_args, sizeof(StepArgs<float>) * 2 * n) == cudaSuccess;
  if (!ok) {
    af_batch_destroy(b);
    return AF_ERR_ALLOC;
  }
  // the persistent pipelined geometry: every grid must allow its staging; the
  // handles' tensor maps (encoded by af_init) go to the device when all have them
  b->pipe_ctas = b->h[0]->pipe_ctas;
  b->pipe_ok = b->pipe_ctas > 0;
  bool tma = true;
  for (int k = 0; k < n && b->pipe_ok; ++k) {
    af_handle* h = b->h[k];
    for (int p = 0; p < 2; ++p) {
      const int cur = h->cur;
      h->cur = p;
      const StepArgs<float> a = step_args<float>(h, 1.0);
      h->cur = cur;
      if (!pipe_eligible(a)) b->pipe_ok = 0;
    }
    tma = tma && h->tma;
  }
  if (b->pipe_ok && tma) {
    for (int p = 0; p < 2 && ok; ++p) {
      ok = cudaMalloc(&b->d_maps[p], sizeof(TileMaps) * n) == cudaSuccess;
      for (int k = 0; k < n && ok; ++k)
        ok = cudaMemcpy(&b->d_maps[p][k], &b->h[k]->tmaps[p], sizeof(TileMaps),
                        cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) {
      af_batch_destroy(b);
      return AF_ERR_ALLOC;
    }
  }
  // AF_BATCH_GEOM=g fixes the geometry instead of timing the candidates
  const char* fg = getenv("AF_BATCH_GEOM");
  if (fg && fg[0] >= '0' && fg[0] < '0' + N_BATCH_GEOMS && !fg[1]) {
    const int g = fg[0] - '0';
    if (!BATCH_GEOMS[g].pipe || b->pipe_ok) {
      b->geom = g;
      for (int q = 0; q < N_BATCH_GEOMS; ++q) b->tune_ms[q] = -1.f;
    }
  }
  *out = b;
  return AF_OK;
}

af_status af_batch_step(af_batch* b, const double* dts, int32_t n_steps) {
  NvtxRange range("af_batch_step");
  if (!b || !dts || n_steps < 0) return AF_ERR_ARG;
  for (int k = 0; k < b->n; ++k) {
    if (!(dts[k] > 0.0)) return AF_ERR_ARG;
    if (b->h[k]->broken) return AF_ERR_STATE;
    af_status prior = map_flags(*(volatile unsigned*)b->h[k]->h_flags);
    if (prior != AF_OK) return prior;
  }
  if (n_steps == 0) return AF_OK;
  DeviceGuard guard(b->h[0]->device);
  // step arguments of both parities, with this call's time steps
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < b->n; ++k) {
      af_handle* h = b->h[k];
      const int cur = h->cur;
      h->cur = p;
      StepArgs<float> a = step_args<float>(h, dts[k]);
      a.prefetch_wave = 0;
      h->cur = cur;
      b->h_args[(size_t)p * b->n + k] = a;
    }
  if (cudaMemcpyAsync(b->d_args, b->h_args, sizeof(StepArgs<float>) * 2 * b->n,
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return AF_ERR_CUDA;
  if (b->geom < 0) {
    af_status st = batch_tune(b);
    if (st != AF_OK) return st;
  }
  const int parity = batch_parity(b);
  if (!b->graph || b->graph_steps != n_steps || b->graph_parity != parity) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaGraph_t g;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return AF_ERR_CUDA;
    }
    int p = parity;
    af_status st = AF_OK;
    for (int s = 0; s < n_steps && st == AF_OK; ++s, p ^= 1) st = batch_launch(b, b->geom, p);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || st != AF_OK) {
      cudaGetLastError();
      return AF_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->graph = nullptr;
      return AF_ERR_CUDA;
    }
    b->graph_steps = n_steps;
    b->graph_parity = parity;
  }
  if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return AF_ERR_CUDA;
  batch_flip(b, n_steps);
  for (int k = 0; k < b->n; ++k)
    cudaMemcpyAsync(b->h[k]->h_flags, b->h[k]->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost,
                    b->stream);
  return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ERR_CUDA;
}

af_status af_batch_sync(af_batch* b) {
  if (!b) return AF_ERR_ARG;
  af_status first = AF_OK;
  for (int k = 0; k < b->n; ++k) {
    af_status st = af_sync(b->h[k]);
    if (first == AF_OK) first = st;
  }
  return first;
}

af_status af_batch_get_state(af_batch* b, int32_t k, const af_state_f64* out, af_memory where) {
  if (!b || k < 0 || k >= b->n) return AF_ERR_ARG;
  return af_get_state(b->h[k], out, where);
}

af_status af_batch_info(af_batch* b, int32_t* geometry, float* tune_ms) {
  if (!b || !geometry) return AF_ERR_ARG;
  *geometry = b->geom;
  if (tune_ms)
    for (int g = 0; g < N_BATCH_GEOMS; ++g) tune_ms[g] = b->tune_ms[g];
  return AF_OK;
}

void af_batch_destroy(af_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (int g = 0; g < N_BATCH_GEOMS; ++g)
    if (b->d_tiles[g]) cudaFree(b->d_tiles[g]);
  for (int p = 0; p < 2; ++p)
    if (b->d_maps[p]) cudaFree(b->d_maps[p]);
  if (b->d_args) cudaFree(b->d_args);
  if (b->h_args) cudaFreeHost(b->h_args);
  if (b->snapshot) cudaFree(b->snapshot);
  if (b->h) {
    for (int k = 0; k < b->n; ++k) af_destroy(b->h[k]);
    delete[] b->h;
  }
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
