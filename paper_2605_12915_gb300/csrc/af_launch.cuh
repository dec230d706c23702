// af_launch.cuh -- host side of the fused step: launch configuration, the
// pipelined kernel's eligibility and tensor maps, and the batched launch.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "af_fused.cuh"

namespace af {

// Raises kernel KERN's dynamic shared-memory limit to `bytes` on the current
// device (the attribute belongs to the device: it is set once per device).
template <auto KERN>
inline cudaError_t allow_smem(size_t bytes) {
  constexpr int MAX_DEVICES = 64;
  static bool done[MAX_DEVICES] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < MAX_DEVICES && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev >= 0 && dev < MAX_DEVICES) done[dev] = true;
  return e;
}

// The pipelined kernel's conditions on the grid and the input planes.
inline bool pipe_eligible(const StepArgs<float>& a) {
  if ((a.nx & 3) != 0 || a.nx < FUSED_TX + 8 || a.ny < FUSED_TY + 6) return false;
  uintptr_t bits = 0;
  for (int q = 0; q < 4; ++q) bits |= (uintptr_t)a.in.avg[q] | (uintptr_t)a.in.lo[q];
  for (int f = 0; f < 3; ++f)
    for (int k = 0; k < 4; ++k) bits |= (uintptr_t)a.in.pt[f][k];
  return (bits & 15) == 0;
}

// Encodes the tensor maps of the 20 input planes in `a` (row-major nx x ny
// floats, staging box of the fused tile geometry); false if the driver lacks the
// encoder or rejects a map.
inline bool encode_tile_maps(const StepArgs<float>& a, TileMaps* out) {
  typedef CUresult (*Encode)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                             const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                             const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    enc = (Encode)fn;
  }
  using G = FusedGeom<FUSED_TX, FUSED_TY>;
  const cuuint64_t dims[2] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny};
  const cuuint64_t strides[1] = {(cuuint64_t)a.nx * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)G::SW, (cuuint32_t)G::CH}, unit[2] = {1, 1};
  for (int p = 0; p < 20; ++p) {
    float* base = p < 12 ? a.in.pt[p >> 2][p & 3] : p < 16 ? a.in.avg[p - 12] : a.in.lo[p - 16];
    if (enc(&out->m[p], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, unit,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// One step of the grid described by `a`: the persistent pipelined kernel on
// `ctas` CTAs when `pipe` is set and the grid allows it (tensor-copy staging
// when `maps` is given), else one CTA per tile.  INTER (pipelined kernel
// only) also stores the intermediates the adjoint needs.
template <bool COMP, bool INTER = false>
inline cudaError_t launch_fused_step(cudaStream_t s, const StepArgs<float>& a, bool pipe,
                                     int ctas, const TileMaps* maps) {
  using G = FusedGeom<FUSED_TX, FUSED_TY>;
  const int tcols = (a.nx + FUSED_TX - 1) / FUSED_TX, trows = (a.ny + FUSED_TY - 1) / FUSED_TY;
  if (pipe && ctas > 0 && pipe_eligible(a)) {
    constexpr auto kern = k_fused_step_pipe<FUSED_TX, FUSED_TY, FUSED_NT, AF_FUSED_MINB, COMP, INTER>;
    const cudaError_t e = allow_smem<kern>(G::SMEM_PIPE);
    if (e != cudaSuccess) return e;
    static TileMaps none;
    const int ntiles = tcols * trows;
    kern<<<ntiles < ctas ? ntiles : ctas, FUSED_NT, G::SMEM_PIPE, s>>>(a, maps ? *maps : none,
                                                                         maps ? 1 : 0);
    return cudaGetLastError();
  }
  if (INTER) return cudaErrorNotSupported;
  constexpr auto kern = k_fused_step<FUSED_TX, FUSED_TY, FUSED_NT, AF_FUSED_MINB, COMP>;
  const cudaError_t e = allow_smem<kern>(G::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grd(tcols, trows);
  kern<<<grd, FUSED_NT, G::SMEM, s>>>(a);
  return cudaGetLastError();
}

// Tile geometries available to the batched launch (the autotuner picks one):
// one CTA per tile of 32x32, 24x16 or 16x16 cells, or (pipe) persistent CTAs
// stepping through the 32x32 tiles with the next tile staged asynchronously.
struct BatchGeometry {
  int tx, ty, nt, minb, pipe;
};
constexpr int N_BATCH_GEOMS = 4;
constexpr BatchGeometry BATCH_GEOMS[N_BATCH_GEOMS] = {
    {32, 32, 512, 1, 0}, {24, 16, 256, 2, 0}, {16, 16, 256, 3, 0},
    {FUSED_TX, FUSED_TY, FUSED_NT, AF_FUSED_MINB, 1}};

template <int TX, int TY, int NT, int MINB, bool COMP>
inline cudaError_t launch_batch_geom(cudaStream_t s, const StepArgs<float>* args,
                                     const int4* tiles, int ntiles) {
  using G = FusedGeom<TX, TY>;
  constexpr auto kern = k_fused_step_batch<TX, TY, NT, MINB, COMP>;
  const cudaError_t e = allow_smem<kern>(G::SMEM);
  if (e != cudaSuccess) return e;
  kern<<<ntiles, NT, G::SMEM, s>>>(args, tiles);
  return cudaGetLastError();
}

// The persistent form: `ctas` CTAs over the tile table; maps (device, one
// TileMaps per grid) or null for cp.async staging only.
template <bool COMP>
inline cudaError_t launch_batch_pipe(cudaStream_t s, const StepArgs<float>* args,
                                     const int4* tiles, int ntiles, const TileMaps* maps,
                                     int ctas) {
  using G = FusedGeom<FUSED_TX, FUSED_TY>;
  constexpr auto kern = k_fused_step_batch_pipe<FUSED_TX, FUSED_TY, FUSED_NT, AF_FUSED_MINB, COMP>;
  const cudaError_t e = allow_smem<kern>(G::SMEM_PIPE);
  if (e != cudaSuccess) return e;
  kern<<<ntiles < ctas ? ntiles : ctas, FUSED_NT, G::SMEM_PIPE, s>>>(args, tiles, ntiles, maps);
  return cudaGetLastError();
}

template <bool COMP>
inline cudaError_t launch_batch(int geom, cudaStream_t s, const StepArgs<float>* args,
                                const int4* tiles, int ntiles, const TileMaps* maps, int ctas) {
  switch (geom) {
    case 0: return launch_batch_geom<32, 32, 512, 1, COMP>(s, args, tiles, ntiles);
    case 1: return launch_batch_geom<24, 16, 256, 2, COMP>(s, args, tiles, ntiles);
    case 2: return launch_batch_geom<16, 16, 256, 3, COMP>(s, args, tiles, ntiles);
    default: return launch_batch_pipe<COMP>(s, args, tiles, ntiles, maps, ctas);
  }
}

}  // namespace af
