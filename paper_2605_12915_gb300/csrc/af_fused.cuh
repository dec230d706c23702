// af_fused.cuh -- the whole RB-TAI / RB step (Sec. 6.1) in one FP32 kernel.
//
// Each CTA owns TX x TY cells.  Everything a step needs around them is staged
// in shared memory, one plane per node family, indexed by cell:
//   W   time-n values float4 (u, v, rho~, p~) of the vertex, x-edge, y-edge and
//       centre families of cells [i0-2, i0+TX+4) x [j0-2, j0+TY+4); the centre
//       family is filled by this CTA's Simpson inversion (phase 1).
//   D   acoustic increments (du, dv, dp) of every family for tau = dt/2 and
//       tau = dt, cells [i0-1, i0+TX+3): every node of every cell that a
//       convective foot can reach (phase 2).
// Phase 0 gathers the tile's input: in the one-tile-per-CTA kernels every
// global load is issued at once (the averages wait in D until phase 1); in the
// persistent kernel the raw planes of the next tile are copied into D while the
// current tile finishes (2D tensor copies completing on an mbarrier, or 16-byte
// cp.async on the periodic boundary), so phase 0 only waits for them and
// converts them into W.  Phase 3 evaluates the two-Picard foot and the
// transported (or additive) point update of the points of cells
// [i0, i0+TX] x [j0, j0+TY] for both durations; the half-step values never
// leave the SM.  Phase 4 forms the space-time Simpson edge fluxes and updates
// the owned cell averages.  Two variants serve the adjoint: one also stores the
// intermediates it linearises about (centres, increments, half-step points),
// the other stops after phase 3 with D still in shared memory, for the reverse
// sweep of the same tile.
//
// Planes of one family are rows of consecutive cells, so a warp working on 32
// consecutive cells touches consecutive addresses: no bank conflicts, and
// stencil offsets become load immediates.  A convective foot may lie up to one
// cell from its point in each direction; displacements are clamped there and
// flagged, so every shared-memory access stays in bounds whatever the data.
#pragma once

#include <cuda.h>  // CUtensorMap (the maps are encoded on the host)

#include "af_common.cuh"
#include "af_ref_kernels.cuh"

// Tile geometry: TX x TY owned cells, NT threads, MINB CTAs per SM (the
// shared-memory footprint FusedGeom::SMEM must fit MINB times in 228 KB).
#ifndef AF_FUSED_TX
#define AF_FUSED_TX 32
#endif
#ifndef AF_FUSED_TY
#define AF_FUSED_TY 32
#endif
#ifndef AF_FUSED_NT
#define AF_FUSED_NT 512
#endif
#ifndef AF_FUSED_MINB
#define AF_FUSED_MINB 1
#endif
#define AF_FUSED_GEOMETRY_SET 1

namespace af {

template <int TX_, int TY_>
struct FusedGeom {
  static constexpr int TX = TX_, TY = TY_;
  static constexpr int CW = TX + 6, CH = TY + 6;    // W cells [i0-2, i0+TX+4)
  static constexpr int DCW = TX + 4, DCH = TY + 4;  // D cells [i0-1, i0+TX+3)
  static constexpr int PW = TX + 1, PH = TY + 1;    // point cells [i0, i0+TX]
  static constexpr int WPL = CW * CH;               // nodes per W plane
  static constexpr int DPL = DCW * DCH;             // floats per D plane
  static constexpr int PPL = PW * PH;               // nodes per point plane
  static constexpr int NPTS = 3 * PPL;              // points of one duration
  static constexpr int NVE = PW * TY, NHE = TX * PH, NE = NVE + NHE;  // edges
  static constexpr size_t W_BYTES = sizeof(float4) * 4 * WPL;
  static constexpr size_t DS_BYTES = sizeof(float) * 12 * DPL;  // one duration
  static constexpr size_t SMEM = W_BYTES + 2 * DS_BYTES;
  // staged raw input of the pipelined kernel (in the D region): 20 planes
  // (points [f][k], averages, lo words) of rows [j0-2, j0+TY+4) and cells
  // [i0-4, i0+TX+4), row stride SW (16-byte rows)
  // (plane stride SPL rounded up to 128 bytes for the tensor copies)
  static constexpr int SW = TX + 8, SPL = (CH * SW + 31) / 32 * 32;
  static constexpr bool STAGE_FITS = 20 * SPL * sizeof(float) <= 2 * DS_BYTES;
  static constexpr size_t SMEM_PIPE = SMEM + 16;  // + the staging mbarrier
  static_assert(4 * NE * sizeof(float) <= W_BYTES, "fluxes alias W");
  static_assert(3 * PPL * sizeof(float4) <= DS_BYTES, "points of one duration alias its increments");
  static_assert(8 * WPL * sizeof(float) <= 2 * DS_BYTES, "averages wait in the D region");
  static_assert(W_BYTES % 16 == 0 && DS_BYTES % 16 == 0, "float4 alignment");
};

// W plane of family f: W + f WPL (float4 per node: u, v, rho~, p~).
// D block of (duration s, family f) at D + (4 s + f) 3 DPL: a float2 plane of
// (u + du, v + dv) (2 DPL floats), then a float plane of dp (DPL floats).  After phase 3 the points of duration s of family f live at
// PT(s) + f PPL (float4), PT(s) = the start of D(s).  During phases 0-1 the
// averages (and lo words) of the W cells occupy D as 8 planes of WPL floats.

// Loader for the generated stencils: node of family F at W cell index `cell`;
// a lattice offset (dx, dy) in half cells resolves at compile time to a family
// plane and a cell offset.
template <int F, int CW, int WPL>
struct LoadW {
  const float4* W;
  int cell;
  __device__ __forceinline__ PUV<float> operator()(int dx, int dy) const {
    const int ax = ((F == 2 || F == 3) ? 1 : 0) + dx, by = ((F == 1 || F == 3) ? 1 : 0) + dy;
    const int fam = (ax & 1) ? ((by & 1) ? 3 : 2) : ((by & 1) ? 1 : 0);
    const float4 w = W[fam * WPL + cell + (by >> 1) * CW + (ax >> 1)];
    PUV<float> o = {w.w, w.x, w.y};
    return o;
  }
};

__device__ __forceinline__ float clamp1(float d) { return fmaxf(fminf(d, 1.0f), -1.0f); }

// Bounds-checking debug builds (-DAF_BOUNDS_CHECK): the shared-memory indices
// of the fused step (foot cells, stencil and node cells, point, edge and flux
// indices) are checked against [lo, hi) of their region; an index outside
// raises FLAG_BOUNDS (AF_ERR_BOUNDS) and is replaced by lo, so the access stays
// inside and the step completes.  Without the define the check compiles away.
__device__ __forceinline__ int idx_checked(int i, int lo, int hi, unsigned& bad) {
  if (i < lo || i >= hi) {
    bad |= FLAG_BOUNDS;
    return lo;
  }
  return i;
}
#ifdef AF_BOUNDS_CHECK
#define AF_IDX(i, lo, hi) ::af::idx_checked((i), (lo), (hi), bad)
#else
#define AF_IDX(i, lo, hi) (i)
#endif

// Node records of the shared planes (W, and the points of each duration):
// float4 (u, v, rho~, p~), so that (u, v) and (rho~, p~) each fill an aligned
// register pair for the paired FP32 operations (__ffma2_rn, __fmul2_rn,
// __fadd2_rn: two lanes in one instruction, each rounded as the scalar
// operation, so a paired evaluation equals the scalar one bitwise).
__device__ __forceinline__ float4 rec4(float r, float u, float v, float p) {
  return make_float4(u, v, r, p);
}
__device__ __forceinline__ float2 rec_uv(const float4& q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ float2 rec_rp(const float4& q) { return make_float2(q.z, q.w); }
__device__ __forceinline__ Prim<float> prim4(float4 w) {
  Prim<float> p = {w.z, w.x, w.y, w.w};
  return p;
}
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// The nine W nodes of the cell at index c, ordered [b][a] (eta row, xi column).
template <int CW, int WPL>
__device__ __forceinline__ void load_cell(const float4* W, int c, float4 n[9]) {
  n[0] = W[c];                    // V(c)
  n[1] = W[2 * WPL + c];          // E_h(c)
  n[2] = W[c + 1];                // V(c+1)
  n[3] = W[WPL + c];              // E_v(c)
  n[4] = W[3 * WPL + c];          // C(c)
  n[5] = W[WPL + c + 1];          // E_v(c+1)
  n[6] = W[c + CW];               // V(c+row)
  n[7] = W[2 * WPL + c + CW];     // E_h(c+row)
  n[8] = W[c + CW + 1];           // V(c+row+1)
}

#define AF_Q2(n, f, lx, ly)                                                        \
  fmaf((ly)[0], fmaf((lx)[0], (n)[0].f, fmaf((lx)[1], (n)[1].f, (lx)[2] * (n)[2].f)), \
       fmaf((ly)[1], fmaf((lx)[0], (n)[3].f, fmaf((lx)[1], (n)[4].f, (lx)[2] * (n)[5].f)), \
            (ly)[2] * fmaf((lx)[0], (n)[6].f, fmaf((lx)[1], (n)[7].f, (lx)[2] * (n)[8].f))))

// sum_ab l_a(xi) l_b(eta) f_ab over the nine nodes of the cell at index c of a
// set of scalar family planes (V, E_v, E_h, C) with row stride R.
template <int R>
__device__ __forceinline__ float q2_eval(const float* pV, const float* pEv, const float* pEh,
                                         const float* pC, int c, const float lx[3],
                                         const float ly[3]) {
  const float r0 = fmaf(lx[0], pV[c], fmaf(lx[1], pEh[c], lx[2] * pV[c + 1]));
  const float r1 = fmaf(lx[0], pEv[c], fmaf(lx[1], pC[c], lx[2] * pEv[c + 1]));
  const float r2 = fmaf(lx[0], pV[c + R], fmaf(lx[1], pEh[c + R], lx[2] * pV[c + R + 1]));
  return fmaf(ly[0], r0, fmaf(ly[1], r1, ly[2] * r2));
}

// sum_ab l_a(xi) l_b(eta) v_ab of a pair of fields (two lanes) over the nine
// nodes v[] of a cell, ordered as load_cell; lxd, lyd hold each weight in both
// lanes.  Each lane performs the operations of AF_Q2 in the same order.
__device__ __forceinline__ float2 q2_pair(const float2 v[9], const float2 lxd[3],
                                          const float2 lyd[3]) {
  const float2 r0 = __ffma2_rn(lxd[0], v[0], __ffma2_rn(lxd[1], v[1], __fmul2_rn(lxd[2], v[2])));
  const float2 r1 = __ffma2_rn(lxd[0], v[3], __ffma2_rn(lxd[1], v[4], __fmul2_rn(lxd[2], v[5])));
  const float2 r2 = __ffma2_rn(lxd[0], v[6], __ffma2_rn(lxd[1], v[7], __fmul2_rn(lxd[2], v[8])));
  return __ffma2_rn(lyd[0], r0, __ffma2_rn(lyd[1], r1, __fmul2_rn(lyd[2], r2)));
}

// the (u, v) and (rho~, p~) pairs of the nine node records n[] of a cell
__device__ __forceinline__ float2 q2_uv(const float4 n[9], const float2 lxd[3],
                                        const float2 lyd[3]) {
  const float2 v[9] = {rec_uv(n[0]), rec_uv(n[1]), rec_uv(n[2]), rec_uv(n[3]), rec_uv(n[4]),
                       rec_uv(n[5]), rec_uv(n[6]), rec_uv(n[7]), rec_uv(n[8])};
  return q2_pair(v, lxd, lyd);
}
__device__ __forceinline__ float2 q2_rp(const float4 n[9], const float2 lxd[3],
                                        const float2 lyd[3]) {
  const float2 v[9] = {rec_rp(n[0]), rec_rp(n[1]), rec_rp(n[2]), rec_rp(n[3]), rec_rp(n[4]),
                       rec_rp(n[5]), rec_rp(n[6]), rec_rp(n[7]), rec_rp(n[8])};
  return q2_pair(v, lxd, lyd);
}

// the same for a pair of fields held as float2 planes (one load per node)
template <int R>
__device__ __forceinline__ float2 q2_eval2(const float2* pV, const float2* pEv, const float2* pEh,
                                           const float2* pC, int c, const float2 lxd[3],
                                           const float2 lyd[3]) {
  const float2 v[9] = {pV[c],  pEh[c],     pV[c + 1],  pEv[c],         pC[c],
                       pEv[c + 1], pV[c + R], pEh[c + R], pV[c + R + 1]};
  return q2_pair(v, lxd, lyd);
}

// both lanes of each Lagrange weight
__device__ __forceinline__ void dup3(const float l[3], float2 d[3]) {
  d[0] = dup2(l[0]);
  d[1] = dup2(l[1]);
  d[2] = dup2(l[2]);
}

// local coordinates of a point displaced by d (cells) from lattice offset o (0
// or 1 half cell): cell offset (floor) and Lagrange weights.
__device__ __forceinline__ int foot_axis(int o, float d, float l[3]) {
  const float f = fmaf(0.5f, (float)o, d);
  const float fl = floorf(f);
  // the Q2 Lagrange basis at t = 2 (f - fl) - 1, its products as multiply-adds
  const float t = fmaf(2.f, f - fl, -1.f), ht = 0.5f * t;
  l[0] = fmaf(ht, t, -ht);
  l[1] = fmaf(-t, t, 1.f);
  l[2] = fmaf(ht, t, ht);
  return (int)fl;
}

// Work item t of a W x H block of cells, visited as 32-wide row chunks first
// (a warp then reads consecutive addresses of one row: no bank conflicts from
// row ends inside a warp) and the remaining W % 32 columns after them.
template <int W, int H>
__device__ __forceinline__ void chunked_xy(int t, int& x, int& y) {
  constexpr int MW = W / 32 * 32, RW = W - MW;
  if constexpr (RW == 0) {
    x = t % MW;
    y = t / MW;
  } else if constexpr (MW == 0) {
    x = t % W;
    y = t / W;
  } else {
    if (t < MW * H) {
      x = t % MW;
      y = t / MW;
    } else {
      const int u = t - MW * H;
      x = MW + u % RW;
      y = u / RW;
    }
  }
}

// Segments of the acoustic work list: the row chunks (M = W / 32 * 32 columns)
// or the remaining W - M columns of family f's W x H block.
template <int M, int H>
__device__ __forceinline__ bool seg_main(int& u, int f, int& fam, int& dx, int& dy) {
  if constexpr (M > 0) {
    if (u < M * H) {
      fam = f; dx = u % M; dy = u / M;
      return true;
    }
    u -= M * H;
  }
  return false;
}
template <int M, int W, int H>
__device__ __forceinline__ bool seg_rest(int& u, int f, int& fam, int& dx, int& dy) {
  constexpr int R = W - M;
  if constexpr (R > 0) {
    if (u < R * H) {
      fam = f; dx = M + u % R; dy = u / R;
      return true;
    }
    u -= R * H;
  }
  return false;
}

// Acoustic work item t -> (family, D cell): the row chunks of the four
// families (V (TX+4)x(TY+4), E_v (TX+4)x(TY+3), E_h (TX+3)x(TY+4), C
// (TX+3)x(TY+3)) first, each starting at a multiple of 32, then their
// remaining columns.
template <int TX, int TY>
__device__ __forceinline__ void acoustic_item(int t, int& fam, int& dx, int& dy) {
  constexpr int W0 = TX + 4, W1 = TX + 4, W2 = TX + 3, W3 = TX + 3;
  constexpr int H0 = TY + 4, H1 = TY + 3, H2 = TY + 4, H3 = TY + 3;
  constexpr int M0 = W0 / 32 * 32, M1 = W1 / 32 * 32, M2 = W2 / 32 * 32, M3 = W3 / 32 * 32;
  int u = t;
  fam = 3; dx = 0; dy = 0;
  if (seg_main<M0, H0>(u, 0, fam, dx, dy) || seg_main<M1, H1>(u, 1, fam, dx, dy) ||
      seg_main<M2, H2>(u, 2, fam, dx, dy) || seg_main<M3, H3>(u, 3, fam, dx, dy) ||
      seg_rest<M0, W0, H0>(u, 0, fam, dx, dy) || seg_rest<M1, W1, H1>(u, 1, fam, dx, dy) ||
      seg_rest<M2, W2, H2>(u, 2, fam, dx, dy))
    return;
  seg_rest<M3, W3, H3>(u, 3, fam, dx, dy);
}

// Point work item t -> (family, point cell) of three PW x PH families: the row
// chunks of the three families first, then their remaining columns.
template <int PW, int PH>
__device__ __forceinline__ void point_item(int t, int& fam, int& px, int& py) {
  constexpr int MP = PW / 32 * 32, RP = PW - MP;
  if constexpr (MP == 0) {
    fam = t / (PW * PH);
    const int u = t - fam * (PW * PH);
    px = u % PW;
    py = u / PW;
  } else if constexpr (RP == 0) {
    fam = t / (MP * PH);
    const int u = t - fam * (MP * PH);
    px = u % MP;
    py = u / MP;
  } else {
    if (t < 3 * MP * PH) {
      fam = t / (MP * PH);
      const int u = t - fam * (MP * PH);
      px = u % MP;
      py = u / MP;
    } else {
      const int u = t - 3 * MP * PH;
      fam = u / (RP * PH);
      const int v = u - fam * (RP * PH);
      px = MP + v % RP;
      py = v / RP;
    }
  }
}

// index in [-n, 2n) wrapped into [0, n)
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Tensor maps of the 20 input planes of one state buffer, each with the staging
// box (SW x CH floats) of FusedGeom: [0,12) points [f][k], [12,16) averages,
// [16,20) lo words.
struct TileMaps {
  CUtensorMap m[20];
};

// State of the staging pipeline of one CTA.
struct PipeCtx {
  const TileMaps* tm;  // null: every tile is staged by cp.async
  unsigned bar;        // shared address of the staging mbarrier
  unsigned phase;      // tensor stagings completed so far
  int late;            // testing only: the next wait for a staged tile reports a timeout
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Waits for the completion of phase `parity` of the mbarrier at `bar`; gives up
// (false) after `max_ns` nanoseconds or `max_polls` polls.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity,
                                                  unsigned long long max_ns = 50000000ull,
                                                  int max_polls = 1 << 22) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int it = 0; it < max_polls; ++it) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > max_ns) return false;
  }
  return false;
}

// A tile whose staging box lies inside the grid is staged by tensor copies (the
// tensor unit would fill the periodic wrap with zeros).
template <int TX, int TY>
__device__ __forceinline__ bool box_inside(int nx, int ny, int i0, int j0) {
  return i0 >= 4 && j0 >= 2 && i0 + TX + 4 <= nx && j0 + TY + 4 <= ny;
}

// Starts the asynchronous copy of the raw input of tile (i0, j0) into the
// staging layout of FusedGeom at S: 20 (16 without lo words) 2D tensor copies
// issued by thread 0 that complete on the mbarrier, or, for tiles on the
// periodic boundary, 16-byte cp.async copies (one commit group).  Needs nx a
// multiple of 4, 16-byte aligned planes, nx >= TX + 8 and ny >= TY + 6 (one
// periodic wrap at most); a quad of cells never straddles the wrap since i0 - 4
// and nx are multiples of 4.
template <int TX, int TY, int NT, bool COMP>
__device__ __forceinline__ void issue_tile_async(const StepArgs<float>& a, const PipeCtx& pc,
                                                 int i0, int j0, float* S) {
  using G = FusedGeom<TX, TY>;
  static_assert(G::STAGE_FITS, "the staged tile fits the D region");
  constexpr int QW = G::SW / 4, CH = G::CH, NPL = COMP ? 20 : 16;
  const unsigned sbase = smem_addr(S);
  if (pc.tm && box_inside<TX, TY>(a.nx, a.ny, i0, j0)) {
    // lane 0 of each warp issues the copies of planes w, w + NT/32, ...; thread 0
    // also arrives with the byte count (a copy may complete before that: the
    // phase cannot end before the single arrival)
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0 && w < NPL) {
      // the region was last read by generic loads of every thread (ordered by
      // the barrier before this call)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (w == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(pc.bar),
                     "r"((unsigned)(NPL * CH * G::SW * sizeof(float)))
                     : "memory");
#pragma unroll 1
      for (int p = w; p < NPL; p += NT / 32)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"(sbase + 4u * (unsigned)(p * G::SPL)),
            "l"(&pc.tm->m[p]), "r"(i0 - 4), "r"(j0 - 2), "r"(pc.bar)
            : "memory");
    }
    return;
  }
  for (int t = threadIdx.x; t < NPL * CH * QW; t += NT) {
    const int m = t % QW, r = (t / QW) % CH, pl = t / (QW * CH);
    const float* base = pl < 12 ? a.in.pt[pl >> 2][pl & 3]
                      : pl < 16 ? a.in.avg[pl - 12] : a.in.lo[pl - 16];
    const size_t id = (size_t)wrap1(j0 - 2 + r, a.ny) * a.nx + wrap1(i0 - 4 + 4 * m, a.nx);
    const unsigned dst = sbase + 4u * (unsigned)(pl * G::SPL + r * G::SW + 4 * m);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(base + id)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// One tile of the step: the CTA owns cells [i0, i0+TX) x [j0, j0+TY) of the grid
// described by `a`.  (pi0, pj0), if pi0 >= 0, is a later tile, of the same grid
// unless `na` describes another one (with tensor maps `ntm`): its rows are
// prefetched into L2 when `pf` is set (same grid only), and with PIPE its raw
// input is copied asynchronously into the D region once this tile no longer
// needs it.
// With PIPE this tile's own input is already on its way there
// (issue_tile_async); false means the wait for it timed out (flagged).  With
// INTER the tile also stores the intermediates of its owned cells that the
// adjoint linearises about: centres (a.wc), increments (a.inc) and half-step
// points (a.half).  With ADJ it stores the centres and half-step points, keeps
// the increments D in shared memory (the points are not written over them) and
// returns after the point updates, for the adjoint's reverse sweep of the tile.
template <int TX, int TY, int NT, bool COMP, bool PIPE, bool INTER = false, bool ADJ = false>
__device__ __forceinline__ bool fused_tile(const StepArgs<float>& a, PipeCtx& pc, int i0, int j0,
                                           int pi0, int pj0, bool pf,
                                           const StepArgs<float>* na = nullptr,
                                           const TileMaps* ntm = nullptr) {
  using G = FusedGeom<TX, TY>;
  constexpr int CW = G::CW, CH = G::CH, DCW = G::DCW, PW = G::PW;
  constexpr int WPL = G::WPL, DPL = G::DPL, PPL = G::PPL;
  extern __shared__ __align__(16) float4 smem4[];
  float4* W = smem4;
  float* D = reinterpret_cast<float*>(smem4 + 4 * WPL);
  float* FLX = reinterpret_cast<float*>(smem4);  // fluxes overwrite W in phase 4

  const int nx = a.nx, ny = a.ny;
  const Gas<float> gas = a.gas;
  unsigned bad = 0;

  // ---- L2 prefetch of a later tile --------------------------------------------
  {
    if (pf && pi0 >= 0 && (nx & 3) == 0) {
      if (pi0 >= 4 && pj0 >= 2 && pi0 + TX + 4 <= nx && pj0 + CH - 2 <= ny) {
        constexpr int NPF = 20 * CH;  // one 16-byte-aligned row segment per plane and row
        for (int t = threadIdx.x; t < NPF; t += NT) {
          const int plane = t / CH, row = t % CH;
          if (!COMP && plane >= 16) continue;
          const float* base = plane < 4 ? a.in.avg[plane]
                            : plane < 16 ? a.in.pt[(plane - 4) / 4][(plane - 4) % 4]
                                         : a.in.lo[plane - 16];
          const float* src = base + (size_t)(pj0 - 2 + row) * nx + (pi0 - 4);
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src),
                       "r"((unsigned)(sizeof(float) * (TX + 8)))
                       : "memory");
        }
      }
    }
  }

  // ---- phase 0: every global load of the step, cells [i0-2, i0+TX+4)^2 ------
  // PIPE: the input is staged in D already; wait for it and build the point
  // families of W from the staged planes (the averages stay staged for phase 1).
  // Otherwise interior tiles read 16-byte quads of cells [i0-4, i0+TX+4) per
  // row (rows are 16-byte aligned when nx is a multiple of 4), and tiles
  // touching the periodic boundary read cell by cell with wrapped indices.
  if constexpr (PIPE) {
    if (pc.tm && box_inside<TX, TY>(nx, ny, i0, j0)) {
      // (pc.late, testing only: report this wait as timed out without polling)
      const bool late = pc.late || !mbar_wait_bounded(pc.bar, pc.phase & 1u);
      if (__syncthreads_or(late)) {
        // flag the timeout, then drain: the copies in flight target this CTA's
        // shared memory and complete in microseconds, so the CTA waits for them
        // (up to 2 s, 40x the first bound) before it leaves
        if (threadIdx.x == 0) atomicOr(a.flags, FLAG_TIMEOUT);
        mbar_wait_bounded(pc.bar, pc.phase & 1u, 2000000000ull, 1 << 30);
        return false;
      }
      ++pc.phase;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    for (int t = threadIdx.x; t < CW * CH; t += NT) {
      int cx, cy;
      chunked_xy<CW, CH>(t, cx, cy);
      const float* S = D + AF_IDX(cy * G::SW + cx + 2, 0, G::SPL);
      const int w = AF_IDX(cy * CW + cx, 0, WPL);
#pragma unroll
      for (int f = 0; f < 3; ++f)
        W[f * WPL + w] = rec4(S[(4 * f) * G::SPL], S[(4 * f + 1) * G::SPL],
                              S[(4 * f + 2) * G::SPL], S[(4 * f + 3) * G::SPL]);
    }
  } else {
    const bool interior = i0 >= 4 && j0 >= 2 && i0 + TX + 4 <= nx && j0 + CH - 2 <= ny &&
                          (nx & 3) == 0;
    if (interior) {
      constexpr int QW = (TX + 8) / 4;  // quads per row
      static_assert(TX % 4 == 0, "quad loads need TX % 4 == 0");
      for (int t = threadIdx.x; t < QW * CH; t += NT) {
        const int m = t % QW, cy = t / QW;
        const size_t id = (size_t)(j0 - 2 + cy) * nx + (i0 - 4 + 4 * m);
        float4 pv[3][4], av[4], lv[4];
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
          for (int k = 0; k < 4; ++k)
            pv[f][k] = __ldg(reinterpret_cast<const float4*>(a.in.pt[f][k] + id));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          av[q] = __ldg(reinterpret_cast<const float4*>(a.in.avg[q] + id));
          lv[q] = COMP ? __ldg(reinterpret_cast<const float4*>(a.in.lo[q] + id))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int cx = 4 * m + e - 2;  // W column of this cell
          if (cx < 0 || cx >= CW) continue;
          const int w = cy * CW + cx;
          auto comp = [&](const float4& v) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; };
#pragma unroll
          for (int f = 0; f < 3; ++f)
            W[f * WPL + w] = rec4(comp(pv[f][0]), comp(pv[f][1]), comp(pv[f][2]), comp(pv[f][3]));
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            D[q * WPL + w] = comp(av[q]);
            if (COMP) D[(4 + q) * WPL + w] = comp(lv[q]);
          }
        }
      }
    } else {
      for (int t = threadIdx.x; t < CW * CH; t += NT) {
        const int cx = t % CW, cy = t / CW;
        const size_t id = (size_t)wrapi(j0 - 2 + cy, ny) * nx + wrapi(i0 - 2 + cx, nx);
#pragma unroll
        for (int f = 0; f < 3; ++f)
          W[f * WPL + t] = rec4(__ldg(a.in.pt[f][0] + id), __ldg(a.in.pt[f][1] + id),
                                __ldg(a.in.pt[f][2] + id), __ldg(a.in.pt[f][3] + id));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          D[q * WPL + t] = __ldg(a.in.avg[q] + id);
          if (COMP) D[(4 + q) * WPL + t] = __ldg(a.in.lo[q] + id);
        }
      }
    }
  }
  __syncthreads();

  // ---- phase 1: centre recovery of cells [i0-2, i0+TX+3) (Eq. center-node) ----
  // deviation form U_c = Ubar + 1/16 sum_corners (Ubar - U_V) + 1/4 sum_edges (Ubar - U_E)
  // averages of W cell (cx, cy): plane k at D[AB + k APL + cy ARS + cx + AOF]
  constexpr int APL = PIPE ? G::SPL : WPL, ARS = PIPE ? G::SW : CW, AOF = PIPE ? 2 : 0;
  constexpr int AB = PIPE ? 12 * G::SPL : 0;
  for (int t = threadIdx.x; t < (CW - 1) * (CH - 1); t += NT) {
    int cx, cy;
    chunked_xy<CW - 1, CH - 1>(t, cx, cy);
    const int c = AF_IDX(cy * CW + cx, 0, WPL - CW - 1);
    const int ca = AF_IDX(AB + cy * ARS + cx + AOF, AB, AB + APL);
    float ub[4], lo[4], sc[4] = {0.f, 0.f, 0.f, 0.f}, se[4] = {0.f, 0.f, 0.f, 0.f}, uc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ub[k] = D[ca + k * APL];
      lo[k] = COMP ? D[ca + (4 + k) * APL] : 0.f;
    }
    const float4 corners[4] = {W[c], W[c + 1], W[c + CW], W[c + CW + 1]};
    const float4 edges[4] = {W[2 * WPL + c], W[2 * WPL + c + CW], W[WPL + c], W[WPL + c + 1]};
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      float u[4];
      cons_from_stored(prim4(corners[n]), gas, u);
#pragma unroll
      for (int k = 0; k < 4; ++k) sc[k] += (ub[k] - u[k]) + lo[k];
      cons_from_stored(prim4(edges[n]), gas, u);
#pragma unroll
      for (int k = 0; k < 4; ++k) se[k] += (ub[k] - u[k]) + lo[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) uc[k] = (ub[k] + lo[k]) + (0.0625f * sc[k] + 0.25f * se[k]);
    const Prim<float> w = stored_from_cons_inv(uc, gas, __fdividef(1.f, gas.rho_ref + uc[0]));
    if (!(gas.rho_ref + w.r > 0.f && gas.p_ref + w.p > 0.f)) bad |= FLAG_NONPHYSICAL;
    W[3 * WPL + c] = rec4(w.r, w.u, w.v, w.p);
    if constexpr (INTER || ADJ) {
      const int gi = i0 - 2 + cx, gj = j0 - 2 + cy;
      if (cx >= 2 && cx < TX + 2 && cy >= 2 && cy < TY + 2 && gi < nx && gj < ny) {
        const size_t id = (size_t)gj * nx + gi;
        a.wc[0][id] = w.r;
        a.wc[1][id] = w.u;
        a.wc[2][id] = w.v;
        a.wc[3][id] = w.p;
      }
    }
  }
  __syncthreads();

  // ---- phase 2: acoustic increments (Sec. 6.1 step 1) -------------------------
  // D cells: V [0,TX+4)x[0,TY+4), E_v [0,TX+4)x[0,TY+3), E_h [0,TX+3)x[0,TY+4),
  // C [0,TX+3)x[0,TY+3); D cell (dx, dy) is W cell (dx+1, dy+1).
  {
    constexpr int nV = (TX + 4) * (TY + 4), nEv = (TX + 4) * (TY + 3),
                  nEh = (TX + 3) * (TY + 4), nC = (TX + 3) * (TY + 3);
    const float dth = a.dt / a.h;
    for (int t = threadIdx.x; t < nV + nEv + nEh + nC; t += NT) {
      int fam, dx, dy;
      acoustic_item<TX, TY>(t, fam, dx, dy);
      // (the stencils reach one cell around wc in every family plane)
      const int wc = AF_IDX((dy + 1) * CW + (dx + 1), CW + 1, WPL - CW - 1);
      const int dc = AF_IDX(dy * DCW + dx, 0, DPL);
      const float4 wk = W[fam * WPL + wc];
      const float rk = gas.rho_ref + wk.z, pk = gas.p_ref + wk.w;
      if (!(rk > 0.f && pk > 0.f)) bad |= FLAG_NONPHYSICAL;
      // Z^2 = gamma p rho, c = gamma p / Z: one reciprocal square root (2 ulp)
      const float gp = gas.gamma * pk, z2 = gp * rk;
      const float Zinv = rsqrtf(z2), Z = z2 * Zinv, c = gp * Zinv;
      const float r1 = c * dth;
      if (r1 > 0.5f) bad |= FLAG_CFL;
      float Gp[3][4], Guv[3][4];
      if (fam == 0) {
        LoadW<0, CW, WPL> ld = {W, wc};
        af_sac_V<float>(ld, wk.w, wk.x, wk.y, Gp, Guv);
      } else if (fam == 1) {
        LoadW<1, CW, WPL> ld = {W, wc};
        af_sac_EV<float>(ld, wk.w, wk.x, wk.y, Gp, Guv);
      } else if (fam == 2) {
        LoadW<2, CW, WPL> ld = {W, wc};
        af_sac_EH<float>(ld, wk.w, wk.x, wk.y, Gp, Guv);
      } else {
        LoadW<3, CW, WPL> ld = {W, wc};
        af_sac_C<float>(ld, wk.w, wk.x, wk.y, Gp, Guv);
      }
      // stored: the acoustically evolved velocity u + du, v + dv and the
      // pressure increment dp (the velocity increments are only ever added to
      // the interpolated velocity, so they are interpolated together with it)
      // r-polynomial coefficients of (du, dv, dp), shared by both durations
      // (the same operations as increments_at)
      float cu[4], cv[4], cp[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        cp[q] = fmaf(Z, Guv[0][q], Gp[0][q]);
        cu[q] = fmaf(Zinv, Gp[1][q], Guv[1][q]);
        cv[q] = fmaf(Zinv, Gp[2][q], Guv[2][q]);
      }
      auto horner = [&](float r, float d[3]) {
        d[2] = r * fmaf(r, fmaf(r, fmaf(r, cp[3], cp[2]), cp[1]), cp[0]);
        d[0] = r * fmaf(r, fmaf(r, fmaf(r, cu[3], cu[2]), cu[1]), cu[0]);
        d[1] = r * fmaf(r, fmaf(r, fmaf(r, cv[3], cv[2]), cv[1]), cv[0]);
      };
      float d[3];
      float2* D0 = reinterpret_cast<float2*>(D + fam * 3 * DPL) + dc;
      float2* D1 = reinterpret_cast<float2*>(D + (4 + fam) * 3 * DPL) + dc;
      float* D0p = D + fam * 3 * DPL + 2 * DPL + dc;
      float* D1p = D + (4 + fam) * 3 * DPL + 2 * DPL + dc;
      // owned node (for the stored intermediates)
      const int gi = i0 - 1 + dx, gj = j0 - 1 + dy;
      const bool own = INTER && dx >= 1 && dx <= TX && dy >= 1 && dy <= TY && gi < nx && gj < ny;
      const size_t gid = own ? (size_t)gj * nx + gi : 0;
      horner(0.5f * r1, d);
      *D0 = make_float2(wk.x + d[0], wk.y + d[1]);
      *D0p = d[2];
      if (own)
        for (int k = 0; k < 3; ++k) a.inc[0][fam][k][gid] = d[k];
      horner(r1, d);
      *D1 = make_float2(wk.x + d[0], wk.y + d[1]);
      *D1p = d[2];
      if (own)
        for (int k = 0; k < 3; ++k) a.inc[1][fam][k][gid] = d[k];
    }
  }
  __syncthreads();

  // ---- phase 3: point updates of cells [i0, i0+TX] x [j0, j0+TY] -------------
  // duration by duration; the points of duration s replace D(s) once every
  // thread is done reading it.  The nine nodes of the first Picard stage's
  // cell are loaded once and reused for the foot when it lies in the same cell.
  // (ADJ: the owned points only, the ones the reverse sweep reads; the others
  // serve the edge fluxes, which ADJ does not form)
  constexpr int NPTS = ADJ ? 3 * TX * TY : G::NPTS;
  constexpr int PER = (NPTS + NT - 1) / NT;
  const float th_full = a.dt / a.h;
#pragma unroll 1
  for (int s = 0; s < 2; ++s) {
    const float th = s == 0 ? 0.5f * th_full : th_full;
    const float* Ds = D + s * 12 * DPL;
    float4 res[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int t = threadIdx.x + k * NT;
      if (k >= NPTS / NT && t >= NPTS) break;  // rounds k < NPTS / NT are full (NT threads)
      int fam, px, py;
      if constexpr (ADJ) {
        fam = t / (TX * TY);
        const int u = t - fam * (TX * TY);
        px = u % TX;
        py = u / TX;
      } else {
        point_item<PW, G::PH>(t, fam, px, py);
      }
      const int ox = fam == 2 ? 1 : 0, oy = fam == 1 ? 1 : 0;
      const int wcP = AF_IDX((py + 2) * CW + (px + 2), 0, WPL);  // W cell of the point's cell
      const float4 wp = W[fam * WPL + wcP];
      // first Picard stage from the point's own velocity (Eq. adv-footpoint)
      const float2 d1 = __fmul2_rn(dup2(-th), rec_uv(wp));
      if (!(fabsf(d1.x) <= 1.f && fabsf(d1.y) <= 1.f)) bad |= FLAG_REACH;
      float lx[3], ly[3];
      float2 lxd[3], lyd[3];
      int ix = foot_axis(ox, clamp1(d1.x), lx), iy = foot_axis(oy, clamp1(d1.y), ly);
      dup3(lx, lxd);
      dup3(ly, lyd);
      // (a cell's nine nodes reach one row and one column beyond it)
      const int c1 = AF_IDX(wcP + iy * CW + ix, 0, WPL - CW - 1);
      float4 n[9];
      load_cell<CW, WPL>(W, c1, n);
      const float2 uv1 = q2_uv(n, lxd, lyd);
      // the foot
      const float2 df = __fmul2_rn(dup2(-th), uv1);
      if (!(fabsf(df.x) <= 1.f && fabsf(df.y) <= 1.f)) bad |= FLAG_REACH;
      ix = foot_axis(ox, clamp1(df.x), lx);
      iy = foot_axis(oy, clamp1(df.y), ly);
      dup3(lx, lxd);
      dup3(ly, lyd);
      const int c2 = AF_IDX(wcP + iy * CW + ix, 0, WPL - CW - 1);
      if (c2 != c1) load_cell<CW, WPL>(W, c2, n);
      const float2 rpf = q2_rp(n, lxd, lyd);  // rho~_f, p~_f
      const float rft = rpf.x, pft = rpf.y;
      Prim<float> nw;
      if (a.variant == 0) {
        // transported increment at the foot; rho from dp / c_f^2 (Sec. 6.1 step 4):
        // u_f + du_f = I_h(u + du)(P_f) since both interpolants share the basis
        const int dcf = AF_IDX((py + 1 + iy) * DCW + (px + 1 + ix), 0, DPL - DCW - 1);
        const float2 e01 = q2_eval2<DCW>(reinterpret_cast<const float2*>(Ds),
                                         reinterpret_cast<const float2*>(Ds + 3 * DPL),
                                         reinterpret_cast<const float2*>(Ds + 6 * DPL),
                                         reinterpret_cast<const float2*>(Ds + 9 * DPL), dcf, lxd,
                                         lyd);
        const float e2 =
            q2_eval<DCW>(Ds + 2 * DPL, Ds + 5 * DPL, Ds + 8 * DPL, Ds + 11 * DPL, dcf, lx, ly);
        const float rf = gas.rho_ref + rft, pf = gas.p_ref + pft;
        if (!(rf > 0.f && pf > 0.f)) bad |= FLAG_NONPHYSICAL;
        nw.r = rft + __fdividef(e2 * rf, gas.gamma * pf);
        nw.u = e01.x;
        nw.v = e01.y;
        nw.p = pft + e2;
      } else {
        // additive update (Eq. barsukow-additive), acoustic rho closure at P
        const int dcp = AF_IDX((py + 1) * DCW + (px + 1), 0, DPL);
        const float2 uv = reinterpret_cast<const float2*>(Ds + fam * 3 * DPL)[dcp];
        const float du = uv.x - wp.x;
        const float dv = uv.y - wp.y;
        const float dp = Ds[(fam * 3 + 2) * DPL + dcp];
        nw.r = rft + __fdividef(dp * (gas.rho_ref + wp.z), gas.gamma * (gas.p_ref + wp.w));
        const float2 uvf = q2_uv(n, lxd, lyd);
        nw.u = uvf.x + du;
        nw.v = uvf.y + dv;
        nw.p = pft + dp;
      }
      if (!(isfinite(nw.r) && isfinite(nw.u) && isfinite(nw.v) && isfinite(nw.p)))
        bad |= FLAG_NONFINITE;
      res[k] = rec4(nw.r, nw.u, nw.v, nw.p);
      // owned points at t^{n+1} go straight to HBM
      const int gi = i0 + px, gj = j0 + py;
      if ((INTER || ADJ) && s == 0 && px < TX && py < TY && gi < nx && gj < ny) {
        const size_t id = (size_t)gj * nx + gi;
        a.half[fam][0][id] = nw.r;
        a.half[fam][1][id] = nw.u;
        a.half[fam][2][id] = nw.v;
        a.half[fam][3][id] = nw.p;
      }
      if (s == 1 && px < TX && py < TY && gi < nx && gj < ny) {
        const size_t id = (size_t)gj * nx + gi;
        a.out.pt[fam][0][id] = nw.r;
        a.out.pt[fam][1][id] = nw.u;
        a.out.pt[fam][2][id] = nw.v;
        a.out.pt[fam][3][id] = nw.p;
      }
    }
    __syncthreads();  // D(s) is dead from here (except for ADJ)
    if constexpr (!ADJ) {
      float4* P = reinterpret_cast<float4*>(D + s * 12 * DPL);
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int t = threadIdx.x + k * NT;
        if (k >= NPTS / NT && t >= NPTS) break;
        int fam, px, py;
        point_item<PW, G::PH>(t, fam, px, py);
        P[AF_IDX(fam * PPL + py * PW + px, 0, 3 * PPL)] = res[k];
      }
    }
  }
  __syncthreads();
  if constexpr (ADJ) {
    if (bad) atomicOr(a.flags, bad);
    return true;
  }

  // ---- phase 4: space-time Simpson fluxes (Sec. 3.1) and average update -------
  // vertical edges (i0+ex, j0+ey), ex in [0, TX], ey in [0, TY); horizontal edges
  // ex in [0, TX), ey in [0, TY].  Computed into registers, then stored over W.
  constexpr int NVE = G::NVE, NE = G::NE;
  constexpr int PERE = (NE + NT - 1) / NT;
  // the owned averages (and lo words) at t^n, loaded while the fluxes are formed
  constexpr int PERC = (TX * TY + NT - 1) / NT;
  float hv[PERC][4], lv[PERC][4];
#pragma unroll
  for (int k = 0; k < PERC; ++k) {
    const int t = threadIdx.x + k * NT;
    const int gi = i0 + t % TX, gj = j0 + t / TX;
    const bool own = t < TX * TY && gi < nx && gj < ny;
    const size_t id = own ? (size_t)gj * nx + gi : 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      hv[k][q] = own ? __ldg(a.in.avg[q] + id) : 0.f;
      lv[k][q] = (COMP && own) ? __ldg(a.in.lo[q] + id) : 0.f;
    }
  }
  float flux[PERE][4];
  const float lam = a.dt / (36.f * a.h);
#pragma unroll
  for (int k = 0; k < PERE; ++k) {
    const int t = threadIdx.x + k * NT;
    if (k >= NE / NT && t >= NE) break;  // rounds k < NE / NT are full (NT threads)
    const bool vert = t < NVE;
    int ex, ey;  // row chunks of each edge family first
    if (vert)
      chunked_xy<PW, TY>(t, ex, ey);
    else
      chunked_xy<TX, G::PH>(t - NVE, ex, ey);
    const int fm = vert ? 1 : 2;              // E_v or E_h
    const int wa = AF_IDX((ey + 2) * CW + (ex + 2), 0, WPL - CW);  // W cell of V(ex, ey)
    const int wb = vert ? wa + CW : wa + 1;   // the edge's other vertex
    const int pa = AF_IDX(ey * PW + ex, 0, vert ? PPL - PW : PPL - 1);
    const int pb = vert ? pa + PW : pa + 1;
    float F[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      Prim<float> xa, xm, xb;
      if (s == 0) {
        xa = prim4(W[wa]);
        xm = prim4(W[fm * WPL + wa]);
        xb = prim4(W[wb]);
      } else {
        const float4* P = reinterpret_cast<const float4*>(D + (s - 1) * 12 * DPL);
        xa = prim4(P[pa]);
        xm = prim4(P[fm * PPL + pa]);
        xb = prim4(P[pb]);
      }
      float fa[4], fmid[4], fb[4];
      if (vert) {
        flux_x(xa, gas, fa);
        flux_x(xm, gas, fmid);
        flux_x(xb, gas, fb);
      } else {
        flux_y(xa, gas, fa);
        flux_y(xm, gas, fmid);
        flux_y(xb, gas, fb);
      }
      const float wt = s == 1 ? 4.f : 1.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) F[q] = fmaf(wt, fmaf(4.f, fmid[q], fa[q] + fb[q]), F[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) flux[k][q] = lam * F[q];
  }
  __syncthreads();  // W and D are dead from here
  // the next tile's input streams into D while the fluxes and averages are stored
  if constexpr (PIPE) {
    if (pi0 >= 0) {
      if (na) {
        PipeCtx q = pc;
        q.tm = ntm;
        issue_tile_async<TX, TY, NT, COMP>(*na, q, pi0, pj0, D);
      } else {
        issue_tile_async<TX, TY, NT, COMP>(a, pc, pi0, pj0, D);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < PERE; ++k) {
    const int t = threadIdx.x + k * NT;
    if (k >= NE / NT && t >= NE) break;
    int ex, ey, e;  // vertical edge ey PW + ex, horizontal NVE + ey TX + ex
    if (t < NVE) {
      chunked_xy<PW, TY>(t, ex, ey);
      e = ey * PW + ex;
    } else {
      chunked_xy<TX, G::PH>(t - NVE, ex, ey);
      e = NVE + ey * TX + ex;
    }
    e = AF_IDX(e, 0, NE);
#pragma unroll
    for (int q = 0; q < 4; ++q) FLX[q * NE + e] = flux[k][q];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PERC; ++k) {
    const int t = threadIdx.x + k * NT;
    const int cx = t % TX, cy = t / TX;
    const int gi = i0 + cx, gj = j0 + cy;
    if (t >= TX * TY || gi >= nx || gj >= ny) continue;
    const size_t id = (size_t)gj * nx + gi;
    const int fl = AF_IDX(cy * PW + cx, 0, NVE - 1), fr = fl + 1;  // vertical edges x_i, x_{i+1}
    const int gb = AF_IDX(NVE + cy * TX + cx, NVE, NE - TX), gt = gb + TX;  // horizontal y_j, y_{j+1}
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float* Fq = FLX + q * NE;
      if (COMP) {
        float hi = hv[k][q], lo = lv[k][q];
        comp_update(hi, lo, Fq[fl], Fq[fr], Fq[gb], Fq[gt]);
        a.out.avg[q][id] = hi;
        a.out.lo[q][id] = lo;
        if (!isfinite(hi)) bad |= FLAG_NONFINITE;
      } else {
        const float v = hv[k][q] - (Fq[fr] - Fq[fl]) - (Fq[gt] - Fq[gb]);
        a.out.avg[q][id] = v;
        if (!isfinite(v)) bad |= FLAG_NONFINITE;
      }
    }
  }
  if (bad) atomicOr(a.flags, bad);
  return true;
}

template <int TX, int TY, int NT, int MINB, bool COMP>
__global__ void __launch_bounds__(NT, MINB)
    k_fused_step(const __grid_constant__ StepArgs<float> a) {
  // prefetch into L2 the tile of the CTA that starts one wave later
  int pi0 = -1, pj0 = -1;
  const int nxt = blockIdx.y * gridDim.x + blockIdx.x + a.prefetch_wave;
  if (a.prefetch_wave > 0 && nxt < gridDim.x * gridDim.y) {
    pi0 = (nxt % gridDim.x) * TX;
    pj0 = (nxt / gridDim.x) * TY;
  }
  PipeCtx none = {nullptr, 0u, 0u};
  fused_tile<TX, TY, NT, COMP, false>(a, none, blockIdx.x * TX, blockIdx.y * TY, pi0, pj0,
                                      pi0 >= 0);
}

// Persistent pipelined form: CTA b steps through tiles b, b + G, b + 2G, ...
// (G = gridDim.x, row-major tile order).  The raw input of its next tile is
// copied into shared memory (tensor copies when `use_tma` and the box lies
// inside the grid, else cp.async after an L2 prefetch at the start of the
// tile) while the current tile stores its averages.  Requires the conditions
// of issue_tile_async.
template <int TX, int TY, int NT, int MINB, bool COMP, bool INTER>
__global__ void __launch_bounds__(NT, MINB)
    k_fused_step_pipe(const __grid_constant__ StepArgs<float> a,
                      const __grid_constant__ TileMaps tm, int use_tma) {
  using G = FusedGeom<TX, TY>;
  extern __shared__ __align__(16) float4 smem4[];
  float* S = reinterpret_cast<float*>(smem4 + 4 * G::WPL);
  PipeCtx pc;
  // tensor copies want 128-byte aligned destinations
  pc.tm = (use_tma && G::W_BYTES % 128 == 0 && (smem_addr(smem4) & 127u) == 0) ? &tm : nullptr;
  pc.bar = smem_addr(reinterpret_cast<char*>(smem4) + G::SMEM);
  pc.phase = 0;
  pc.late = a.late_first_wait;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pc.bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (pc.tm && (threadIdx.x & 31) == 0)
    for (int p = threadIdx.x >> 5; p < 20; p += NT / 32)
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tm.m[p]) : "memory");
  __syncthreads();
  const int tcols = (a.nx + TX - 1) / TX, ntiles = tcols * ((a.ny + TY - 1) / TY);
  int tile = blockIdx.x;
  if (tile < ntiles)
    issue_tile_async<TX, TY, NT, COMP>(a, pc, (tile % tcols) * TX, (tile / tcols) * TY, S);
  for (; tile < ntiles; tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    const int pi0 = nxt < ntiles ? (nxt % tcols) * TX : -1, pj0 = (nxt / tcols) * TY;
    // (an L2 prefetch only pays for cp.async staging; tensor copies are fast enough)
    if (!fused_tile<TX, TY, NT, COMP, true, INTER>(a, pc, (tile % tcols) * TX,
                                                   (tile / tcols) * TY, pi0, pj0,
                                                   a.prefetch_wave > 0 && !pc.tm))
      break;
  }
}

// Batched form: one CTA per entry (grid, i0, j0, -) of a tile table spanning
// many independent grids; args[grid] describes each grid's step.
template <int TX, int TY, int NT, int MINB, bool COMP>
__global__ void __launch_bounds__(NT, MINB)
    k_fused_step_batch(const StepArgs<float>* __restrict__ args, const int4* __restrict__ tiles) {
  const int4 t = tiles[blockIdx.x];
  PipeCtx none = {nullptr, 0u, 0u};
  fused_tile<TX, TY, NT, COMP, false>(args[t.x], none, t.y, t.z, -1, -1, false);
}

// Batched persistent pipelined form: CTA b steps through entries b, b + G, ...
// of the tile table (G = gridDim.x); the raw input of its next tile, of
// whichever grid, is staged while the current one stores its averages.  maps,
// if not null, holds the tensor maps of every grid's current input planes
// (maps[grid]); every grid meets the conditions of issue_tile_async.
template <int TX, int TY, int NT, int MINB, bool COMP>
__global__ void __launch_bounds__(NT, MINB)
    k_fused_step_batch_pipe(const StepArgs<float>* __restrict__ args,
                            const int4* __restrict__ tiles, int ntiles,
                            const TileMaps* __restrict__ maps) {
  using G = FusedGeom<TX, TY>;
  extern __shared__ __align__(16) float4 smem4[];
  float* S = reinterpret_cast<float*>(smem4 + 4 * G::WPL);
  const bool tma = maps && G::W_BYTES % 128 == 0 && (smem_addr(smem4) & 127u) == 0;
  PipeCtx pc;
  pc.tm = nullptr;
  pc.bar = smem_addr(reinterpret_cast<char*>(smem4) + G::SMEM);
  pc.phase = 0;
  pc.late = 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pc.bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int t = blockIdx.x;
  if (t < ntiles) {
    const int4 e = tiles[t];
    pc.tm = tma ? &maps[e.x] : nullptr;
    issue_tile_async<TX, TY, NT, COMP>(args[e.x], pc, e.y, e.z, S);
  }
  for (; t < ntiles; t += gridDim.x) {
    const int4 e = tiles[t];
    const int nt = t + gridDim.x;
    const int4 ne = nt < ntiles ? tiles[nt] : make_int4(0, -1, -1, 0);
    // the current tile was staged with its own grid's maps
    pc.tm = tma ? &maps[e.x] : nullptr;
    if (!fused_tile<TX, TY, NT, COMP, true>(args[e.x], pc, e.y, e.z, ne.y, ne.z, false,
                                            &args[ne.x], tma ? &maps[ne.x] : nullptr))
      break;
  }
}

constexpr int FUSED_TX = AF_FUSED_TX, FUSED_TY = AF_FUSED_TY, FUSED_NT = AF_FUSED_NT;

}  // namespace af
