// af_fused.cuh -- the whole RB-TAI / RB step (Sec. 6.1) in one FP32 kernel.
//
// Each CTA owns TX x TY cells.  Everything a step needs around them is staged
// in shared memory on the half-cell lattice (see af_common.cuh):
//   LW  time-n primitive values (rho,u,v,p) on the lattice covering cells
//       [i0-2, i0+TX+3) x [j0-2, j0+TY+3); the centre nodes are filled by the
//       Simpson inversion of this CTA (phase 1).
//   LD  acoustic increments (du,dv,dp) for tau = dt/2 and dt on the lattice
//       of every node of every cell a convective foot can reach (phase 2).
// Phase 3 evaluates the two-Picard foot and the transported (or additive)
// point update of the points of cells [i0, i0+TX] x [j0, j0+TY] for both
// durations; the half-step values never leave the SM.  Phase 4 forms the
// space-time Simpson edge fluxes and updates the owned cell averages.
// A convective foot may lie up to one cell from its point in each direction
// (displacements are clamped there and flagged, so shared-memory accesses stay
// in bounds whatever the data).
#pragma once

#include "af_common.cuh"
#include "af_ref_kernels.cuh"

namespace af {

template <int TX_, int TY_>
struct FusedGeom {
  static constexpr int TX = TX_, TY = TY_;
  static constexpr int FW = 2 * TX + 11, FH = 2 * TY + 11;  // LW: fine [2i0-4, 2i0+2TX+6]
  static constexpr int DW = 2 * TX + 7, DH = 2 * TY + 7;    // LD: fine [2i0-2, 2i0+2TX+4]
  static constexpr int PW = TX + 1, PH = TY + 1;            // point cells [i0, i0+TX]
  static constexpr int CW = TX + 6, CH = TY + 6;            // loaded cells [i0-2, i0+TX+4)
  static constexpr int NW = TX + 5, NH = TY + 5;            // centre cells [i0-2, i0+TX+3)
  static constexpr int NPTS = 3 * PW * PH;                 // points of one duration
  static constexpr int LDS = (3 * DW * DH + 3) / 4 * 4;     // floats per duration in LD
  static constexpr size_t LW_BYTES = sizeof(float4) * FW * FH;
  static constexpr size_t LD_BYTES = sizeof(float) * 2 * LDS;
  static constexpr size_t FL_BYTES = sizeof(float) * 4 * (PW * TY + TX * PH);
  static constexpr size_t SMEM = LW_BYTES + LD_BYTES;
  static_assert(FL_BYTES <= LW_BYTES, "fluxes alias the LW region");
  static_assert(4 * NPTS <= LDS, "the points of one duration alias its increments");
};

struct LoadSmem {
  const float4* LW;
  int base;  // index of the node itself
  int fw;
  __device__ __forceinline__ PUV<float> operator()(int dx, int dy) const {
    float4 w = LW[base + dy * fw + dx];
    PUV<float> o = {w.w, w.y, w.z};
    return o;
  }
};

__device__ __forceinline__ Prim<float> as_prim(float4 w) {
  Prim<float> p = {w.x, w.y, w.z, w.w};
  return p;
}

__device__ __forceinline__ float clamp1(float d) { return fmaxf(fminf(d, 1.0f), -1.0f); }

// Q2 evaluation of the four primitives from LW in the cell whose lower-left
// lattice node is `base`.
template <int FW>
__device__ __forceinline__ Prim<float> eval_w_s(const float4* LW, int base, float xi,
                                                float eta) {
  float lx[3], ly[3];
  lagrange3(xi, lx);
  lagrange3(eta, ly);
  Prim<float> s = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    Prim<float> row = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float4 w = LW[base + b * FW + q];
      row.r = fmaf(lx[q], w.x, row.r);
      row.u = fmaf(lx[q], w.y, row.u);
      row.v = fmaf(lx[q], w.z, row.v);
      row.p = fmaf(lx[q], w.w, row.p);
    }
    s.r = fmaf(ly[b], row.r, s.r);
    s.u = fmaf(ly[b], row.u, s.u);
    s.v = fmaf(ly[b], row.v, s.v);
    s.p = fmaf(ly[b], row.p, s.p);
  }
  return s;
}

template <int DW>
__device__ __forceinline__ void eval_d_s(const float* LD, int base, float xi, float eta,
                                         float out[3]) {
  float lx[3], ly[3];
  lagrange3(xi, lx);
  lagrange3(eta, ly);
  out[0] = out[1] = out[2] = 0.f;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    float row[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float* d = LD + 3 * (base + b * DW + q);
#pragma unroll
      for (int k = 0; k < 3; ++k) row[k] = fmaf(lx[q], d[k], row[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) out[k] = fmaf(ly[b], row[k], out[k]);
  }
}

template <int TX, int TY, int NT, bool COMP>
__global__ void __launch_bounds__(NT, 1) k_fused_step(StepArgs<float> a) {
  using G = FusedGeom<TX, TY>;
  constexpr int FW = G::FW, FH = G::FH, DW = G::DW, PW = G::PW, PH = G::PH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* LW = reinterpret_cast<float4*>(smem_raw);
  float* LD = reinterpret_cast<float*>(smem_raw + G::LW_BYTES);  // [2][LDS]: [DH][DW][3]
  // after phase 3 the points of duration s overwrite LD[s]: PT(s) = [3][PH][PW] float4
  auto PT = [&](int s) { return reinterpret_cast<float4*>(LD + s * G::LDS); };
  float* FLX = reinterpret_cast<float*>(smem_raw);                 // fluxes (after LW)

  const int nx = a.nx, ny = a.ny;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  unsigned bad = 0;

  // ---- phase 0: point values of cells [i0-2, i0+TX+4) x [j0-2, j0+TY+4) ------
  for (int t = threadIdx.x; t < G::CW * G::CH; t += NT) {
    const int cx = t % G::CW, cy = t / G::CW;
    const size_t id = (size_t)wrapi(j0 - 2 + cy, ny) * nx + wrapi(i0 - 2 + cx, nx);
    const int lx = 2 * cx, ly = 2 * cy;
    if (ly < FH) {
      if (lx < FW)
        LW[ly * FW + lx] = make_float4(__ldg(a.in.pt[0][0] + id), __ldg(a.in.pt[0][1] + id),
                                       __ldg(a.in.pt[0][2] + id), __ldg(a.in.pt[0][3] + id));
      if (lx + 1 < FW)
        LW[ly * FW + lx + 1] = make_float4(__ldg(a.in.pt[2][0] + id), __ldg(a.in.pt[2][1] + id),
                                           __ldg(a.in.pt[2][2] + id), __ldg(a.in.pt[2][3] + id));
    }
    if (ly + 1 < FH && lx < FW)
      LW[(ly + 1) * FW + lx] = make_float4(__ldg(a.in.pt[1][0] + id), __ldg(a.in.pt[1][1] + id),
                                           __ldg(a.in.pt[1][2] + id), __ldg(a.in.pt[1][3] + id));
  }
  __syncthreads();

  // ---- phase 1: centre recovery of cells [i0-2, i0+TX+3) (Eq. center-node) ----
  for (int t = threadIdx.x; t < G::NW * G::NH; t += NT) {
    const int cx = t % G::NW, cy = t / G::NW;
    const size_t id = (size_t)wrapi(j0 - 2 + cy, ny) * nx + wrapi(i0 - 2 + cx, nx);
    float ub[4], lo[4], c[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f}, uc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ub[k] = __ldg(a.in.avg[k] + id);
      lo[k] = COMP ? __ldg(a.in.lo[k] + id) : 0.f;
    }
    const int b = (2 * cy) * FW + 2 * cx;  // lower-left lattice node of the cell
    const int cidx[4] = {b, b + 2, b + 2 * FW, b + 2 * FW + 2};
    const int eidx[4] = {b + 1, b + 2 * FW + 1, b + FW, b + FW + 2};
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      float u[4];
      cons_from_stored(as_prim(LW[cidx[n]]), a.gas, u);
#pragma unroll
      for (int k = 0; k < 4; ++k) c[k] += (ub[k] - u[k]) + lo[k];
      cons_from_stored(as_prim(LW[eidx[n]]), a.gas, u);
#pragma unroll
      for (int k = 0; k < 4; ++k) e[k] += (ub[k] - u[k]) + lo[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) uc[k] = (ub[k] + lo[k]) + (0.0625f * c[k] + 0.25f * e[k]);
    Prim<float> w = stored_from_cons(uc, a.gas);
    if (!(a.gas.rho_ref + w.r > 0.f && a.gas.p_ref + w.p > 0.f)) bad |= FLAG_NONPHYSICAL;
    LW[b + FW + 1] = make_float4(w.r, w.u, w.v, w.p);
  }
  __syncthreads();

  // ---- phase 2: acoustic increments on LD (Sec. 6.1 step 1) -------------------
  {
    constexpr int nV = (TX + 4) * (TY + 4), nEv = (TX + 4) * (TY + 3),
                  nEh = (TX + 3) * (TY + 4), nC = (TX + 3) * (TY + 3);
    for (int t = threadIdx.x; t < nV + nEv + nEh + nC; t += NT) {
      int fam, dx, dy;
      if (t < nV) {
        fam = 0; dx = 2 * (t % (TX + 4)); dy = 2 * (t / (TX + 4));
      } else if (t < nV + nEv) {
        int u = t - nV; fam = 1; dx = 2 * (u % (TX + 4)); dy = 2 * (u / (TX + 4)) + 1;
      } else if (t < nV + nEv + nEh) {
        int u = t - nV - nEv; fam = 2; dx = 2 * (u % (TX + 3)) + 1; dy = 2 * (u / (TX + 3));
      } else {
        int u = t - nV - nEv - nEh; fam = 3; dx = 2 * (u % (TX + 3)) + 1; dy = 2 * (u / (TX + 3)) + 1;
      }
      const int node = (dy + 2) * FW + (dx + 2);
      const float4 wk4 = LW[node];
      const float rk = a.gas.rho_ref + wk4.x, pk = a.gas.p_ref + wk4.w;
      if (!(rk > 0.f && pk > 0.f)) bad |= FLAG_NONPHYSICAL;
      const float c = sqrtf(a.gas.gamma * pk / rk);
      const float Z = rk * c, Zinv = 1.f / Z;
      const float r1 = c * a.dt / a.h;
      if (r1 > 0.5f) bad |= FLAG_CFL;
      float Gp[3][4], Guv[3][4];
      LoadSmem ld = {LW, node, FW};
      if (fam == 0) af_sac_V<float>(ld, wk4.w, wk4.y, wk4.z, Gp, Guv);
      else if (fam == 1) af_sac_EV<float>(ld, wk4.w, wk4.y, wk4.z, Gp, Guv);
      else if (fam == 2) af_sac_EH<float>(ld, wk4.w, wk4.y, wk4.z, Gp, Guv);
      else af_sac_C<float>(ld, wk4.w, wk4.y, wk4.z, Gp, Guv);
      float d[3];
      float* dst = LD + 3 * (dy * DW + dx);
      increments_at(Gp, Guv, Z, Zinv, 0.5f * r1, d);
      dst[0] = d[0]; dst[1] = d[1]; dst[2] = d[2];
      increments_at(Gp, Guv, Z, Zinv, r1, d);
      dst += G::LDS;
      dst[0] = d[0]; dst[1] = d[1]; dst[2] = d[2];
    }
  }
  __syncthreads();

  // ---- phase 3: point updates of cells [i0, i0+TX] x [j0, j0+TY] -------------
  // duration by duration: the results of duration s replace LD[s] once every
  // thread is done reading it.
  constexpr int NPTS = G::NPTS;
  constexpr int PER = (NPTS + NT - 1) / NT;
  const float th_full = a.dt / a.h;
#pragma unroll 1
  for (int s = 0; s < 2; ++s) {
    const float th = s == 0 ? 0.5f * th_full : th_full;
    const float* LDs = LD + s * G::LDS;
    float4 res[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int t = threadIdx.x + k * NT;
      if (t >= NPTS) break;
      const int fam = t / (PW * PH), rem = t % (PW * PH);
      const int px = rem % PW, py = rem / PW;
      const int ox = fam == 2 ? 1 : 0, oy = fam == 1 ? 1 : 0;
      const int lxp = 2 * px + 4 + ox, lyp = 2 * py + 4 + oy;  // LW coordinates of P
      const float4 wp = LW[lyp * FW + lxp];
      // first Picard stage from the point's own velocity (Eq. adv-footpoint)
      float d1x = -th * wp.y, d1y = -th * wp.z;
      if (!(fabsf(d1x) <= 1.f && fabsf(d1y) <= 1.f)) bad |= FLAG_REACH;
      d1x = clamp1(d1x);
      d1y = clamp1(d1y);
      float fx = 0.5f * ox + d1x, fy = 0.5f * oy + d1y;
      float flx = floorf(fx), fly = floorf(fy);
      const int cb = (lyp - oy + 2 * (int)fly) * FW + (lxp - ox + 2 * (int)flx);
      const Prim<float> w1 = eval_w_s<FW>(LW, cb, 2.f * (fx - flx) - 1.f, 2.f * (fy - fly) - 1.f);
      // the foot
      float dfx = -th * w1.u, dfy = -th * w1.v;
      if (!(fabsf(dfx) <= 1.f && fabsf(dfy) <= 1.f)) bad |= FLAG_REACH;
      dfx = clamp1(dfx);
      dfy = clamp1(dfy);
      fx = 0.5f * ox + dfx;
      fy = 0.5f * oy + dfy;
      flx = floorf(fx);
      fly = floorf(fy);
      const float xi = 2.f * (fx - flx) - 1.f, eta = 2.f * (fy - fly) - 1.f;
      const int fcx = lxp - ox + 2 * (int)flx, fcy = lyp - oy + 2 * (int)fly;  // LW coords
      const Prim<float> wf = eval_w_s<FW>(LW, fcy * FW + fcx, xi, eta);
      float d[3];
      Prim<float> nw;
      if (a.variant == 0) {
        // transported increment at the foot, rho from dp / c_f^2 (Sec. 6.1 step 4)
        eval_d_s<DW>(LDs, (fcy - 2) * DW + (fcx - 2), xi, eta, d);
        const float rf = a.gas.rho_ref + wf.r, pf = a.gas.p_ref + wf.p;
        if (!(rf > 0.f && pf > 0.f)) bad |= FLAG_NONPHYSICAL;
        nw.r = wf.r + d[2] * rf / (a.gas.gamma * pf);
      } else {
        // additive update (Eq. barsukow-additive), acoustic rho closure at P
        const float* dp = LDs + 3 * ((lyp - 2) * DW + (lxp - 2));
        d[0] = dp[0];
        d[1] = dp[1];
        d[2] = dp[2];
        nw.r = wf.r + d[2] * (a.gas.rho_ref + wp.x) / (a.gas.gamma * (a.gas.p_ref + wp.w));
      }
      nw.u = wf.u + d[0];
      nw.v = wf.v + d[1];
      nw.p = wf.p + d[2];
      if (!(isfinite(nw.r) && isfinite(nw.u) && isfinite(nw.v) && isfinite(nw.p)))
        bad |= FLAG_NONFINITE;
      res[k] = make_float4(nw.r, nw.u, nw.v, nw.p);
      // owned points at t^{n+1} go straight to HBM
      const int gi = i0 + px, gj = j0 + py;
      if (s == 1 && px < TX && py < TY && gi < nx && gj < ny) {
        const size_t id = (size_t)gj * nx + gi;
        a.out.pt[fam][0][id] = nw.r;
        a.out.pt[fam][1][id] = nw.u;
        a.out.pt[fam][2][id] = nw.v;
        a.out.pt[fam][3][id] = nw.p;
      }
    }
    __syncthreads();  // LD[s] is dead from here
    float4* P = PT(s);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int t = threadIdx.x + k * NT;
      if (t >= NPTS) break;
      P[t] = res[k];
    }
  }
  __syncthreads();

  // ---- phase 4: space-time Simpson fluxes (Sec. 3.1) and average update -------
  // vertical edges (i0+ex, j0+ey), ex in [0, TX], ey in [0, TY); horizontal edges
  // ex in [0, TX), ey in [0, TY].  Computed into registers, then stored over LW.
  constexpr int NVE = PW * TY, NHE = TX * PH, NE = NVE + NHE;
  constexpr int PERE = (NE + NT - 1) / NT;
  float flux[PERE][4];
  const float lam = a.dt / (36.f * a.h);
#pragma unroll
  for (int k = 0; k < PERE; ++k) {
    const int t = threadIdx.x + k * NT;
    if (t >= NE) break;
    const bool vert = t < NVE;
    const int u = vert ? t : t - NVE;
    const int ex = vert ? u % PW : u % TX, ey = vert ? u / PW : u / TX;
    // time-n nodes from LW, half/full from PT: a = V(ex,ey), m = E_v or E_h, b = next V
    const int la = (2 * ey + 4) * FW + (2 * ex + 4);
    const int lm = vert ? la + FW : la + 1;
    const int lb = vert ? la + 2 * FW : la + 2;
    const int pa = ey * PW + ex;
    const int pm = (vert ? 1 : 2) * PW * PH + pa;
    const int pb = vert ? pa + PW : pa + 1;
    float F[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      Prim<float> wa, wm, wb;
      if (s == 0) {
        wa = as_prim(LW[la]); wm = as_prim(LW[lm]); wb = as_prim(LW[lb]);
      } else {
        const float4* P = PT(s - 1);
        wa = as_prim(P[pa]); wm = as_prim(P[pm]); wb = as_prim(P[pb]);
      }
      float fa[4], fm[4], fb[4];
      if (vert) {
        flux_x(wa, a.gas, fa); flux_x(wm, a.gas, fm); flux_x(wb, a.gas, fb);
      } else {
        flux_y(wa, a.gas, fa); flux_y(wm, a.gas, fm); flux_y(wb, a.gas, fb);
      }
      const float wt = s == 1 ? 4.f : 1.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) F[c] = fmaf(wt, fa[c] + 4.f * fm[c] + fb[c], F[c]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) flux[k][c] = lam * F[c];
  }
  __syncthreads();  // LW is dead from here
#pragma unroll
  for (int k = 0; k < PERE; ++k) {
    const int t = threadIdx.x + k * NT;
    if (t >= NE) break;
#pragma unroll
    for (int c = 0; c < 4; ++c) FLX[c * NE + t] = flux[k][c];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < TX * TY; t += NT) {
    const int cx = t % TX, cy = t / TX;
    const int gi = i0 + cx, gj = j0 + cy;
    if (gi >= nx || gj >= ny) continue;
    const size_t id = (size_t)gj * nx + gi;
    const int fl = cy * PW + cx, fr = fl + 1;            // vertical edges x_i, x_{i+1}
    const int gb = NVE + cy * TX + cx, gt = gb + TX;     // horizontal edges y_j, y_{j+1}
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float* Fc = FLX + c * NE;
      if (COMP) {
        float hi = __ldg(a.in.avg[c] + id), lo = __ldg(a.in.lo[c] + id);
        comp_update(hi, lo, Fc[fl], Fc[fr], Fc[gb], Fc[gt]);
        a.out.avg[c][id] = hi;
        a.out.lo[c][id] = lo;
        if (!isfinite(hi)) bad |= FLAG_NONFINITE;
      } else {
        const float v = __ldg(a.in.avg[c] + id) - (Fc[fr] - Fc[fl]) - (Fc[gt] - Fc[gb]);
        a.out.avg[c][id] = v;
        if (!isfinite(v)) bad |= FLAG_NONFINITE;
      }
    }
  }
  if (bad) atomicOr(a.flags, bad);
}

constexpr int FUSED_TX = 32, FUSED_TY = 32, FUSED_NT = 512;

template <bool COMP>
inline cudaError_t launch_fused_step(cudaStream_t s, const StepArgs<float>& a) {
  using G = FusedGeom<FUSED_TX, FUSED_TY>;
  auto kern = k_fused_step<FUSED_TX, FUSED_TY, FUSED_NT, COMP>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::SMEM);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grd((a.nx + FUSED_TX - 1) / FUSED_TX, (a.ny + FUSED_TY - 1) / FUSED_TY);
  kern<<<grd, FUSED_NT, G::SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace af
