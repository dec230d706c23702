// af_fused.cuh -- the whole RB-TAI / RB step (Sec. 6.1) in one FP32 kernel.
//
// Each CTA owns TX x TY cells.  Everything a step needs around them is staged
// in shared memory, one plane per (node family, component), indexed by cell:
//   W   time-n values (rho~, u, v, p~) of the vertex, x-edge, y-edge and
//       centre families of cells [i0-2, i0+TX+4) x [j0-2, j0+TY+4); the centre
//       family is filled by this CTA's Simpson inversion (phase 1).
//   D   acoustic increments (du, dv, dp) of every family for tau = dt/2 and
//       tau = dt, cells [i0-1, i0+TX+3): every node of every cell that a
//       convective foot can reach (phase 2).
// Phase 3 evaluates the two-Picard foot and the transported (or additive)
// point update of the points of cells [i0, i0+TX] x [j0, j0+TY] for both
// durations; the half-step values never leave the SM.  Phase 4 forms the
// space-time Simpson edge fluxes and updates the owned cell averages.
//
// Planes of one family are rows of consecutive cells, so a warp working on 32
// consecutive cells touches 32 consecutive words: no bank conflicts, and
// stencil offsets become load immediates.  A convective foot may lie up to one
// cell from its point in each direction; displacements are clamped there and
// flagged, so every shared-memory access stays in bounds whatever the data.
#pragma once

#include "af_common.cuh"
#include "af_ref_kernels.cuh"

namespace af {

template <int TX_, int TY_>
struct FusedGeom {
  static constexpr int TX = TX_, TY = TY_;
  static constexpr int CW = TX + 6, CH = TY + 6;    // W cells [i0-2, i0+TX+4)
  static constexpr int DCW = TX + 4, DCH = TY + 4;  // D cells [i0-1, i0+TX+3)
  static constexpr int PW = TX + 1, PH = TY + 1;    // point cells [i0, i0+TX]
  static constexpr int WPL = CW * CH;               // floats per W plane
  static constexpr int DPL = DCW * DCH;             // floats per D plane
  static constexpr int PPL = PW * PH;               // floats per point plane
  static constexpr int NPTS = 3 * PPL;              // points of one duration
  static constexpr int NVE = PW * TY, NHE = TX * PH, NE = NVE + NHE;  // edges
  static constexpr size_t W_BYTES = sizeof(float) * 16 * WPL;
  static constexpr size_t D_BYTES = sizeof(float) * 24 * DPL;
  static constexpr size_t SMEM = W_BYTES + D_BYTES;
  static_assert(4 * NE <= 16 * WPL, "fluxes alias W");
  static_assert(PPL <= DPL, "points of one duration alias its increments");
};

// Plane of W for (family f, component k): W + (4 f + k) WPL, k = rho~, u, v, p~.
// Plane of D for (duration s, family f, component k): D + ((4 s + f) 3 + k) DPL,
// k = du, dv, dp.  After phase 3 the points of duration s, plane (family f,
// component k), live at D + 12 s DPL + (4 f + k) PPL.

// Loader for the generated stencils: node of family F at W cell index `cell`;
// a lattice offset (dx, dy) in half cells resolves at compile time to a family
// plane and a cell offset.
template <int F, int CW, int WPL>
struct LoadW {
  const float* W;
  int cell;
  __device__ __forceinline__ PUV<float> operator()(int dx, int dy) const {
    const int ax = ((F == 2 || F == 3) ? 1 : 0) + dx, by = ((F == 1 || F == 3) ? 1 : 0) + dy;
    const int fam = (ax & 1) ? ((by & 1) ? 3 : 2) : ((by & 1) ? 1 : 0);
    const float* base = W + 4 * fam * WPL + cell + (by >> 1) * CW + (ax >> 1);
    PUV<float> o = {base[3 * WPL], base[WPL], base[2 * WPL]};
    return o;
  }
};

__device__ __forceinline__ float clamp1(float d) { return fmaxf(fminf(d, 1.0f), -1.0f); }

// sum_ab l_a(xi) l_b(eta) f_ab over the nine nodes of the cell at index c of a
// set of family planes (V, E_v, E_h, C) with row stride R.
template <int R>
__device__ __forceinline__ float q2_eval(const float* pV, const float* pEv, const float* pEh,
                                         const float* pC, int c, const float lx[3],
                                         const float ly[3]) {
  const float r0 = fmaf(lx[0], pV[c], fmaf(lx[1], pEh[c], lx[2] * pV[c + 1]));
  const float r1 = fmaf(lx[0], pEv[c], fmaf(lx[1], pC[c], lx[2] * pEv[c + 1]));
  const float r2 = fmaf(lx[0], pV[c + R], fmaf(lx[1], pEh[c + R], lx[2] * pV[c + R + 1]));
  return fmaf(ly[0], r0, fmaf(ly[1], r1, ly[2] * r2));
}

template <int TX, int TY, int NT, bool COMP>
__global__ void __launch_bounds__(NT, 1) k_fused_step(StepArgs<float> a) {
  using G = FusedGeom<TX, TY>;
  constexpr int CW = G::CW, CH = G::CH, DCW = G::DCW, PW = G::PW;
  constexpr int WPL = G::WPL, DPL = G::DPL, PPL = G::PPL;
  extern __shared__ __align__(16) float smem[];
  float* W = smem;
  float* D = smem + 16 * WPL;
  float* FLX = smem;  // fluxes overwrite W in phase 4

  const int nx = a.nx, ny = a.ny;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const Gas<float> gas = a.gas;
  unsigned bad = 0;

  // ---- phase 0: point values of cells [i0-2, i0+TX+4) x [j0-2, j0+TY+4) ------
  {
    const bool interior = i0 >= 2 && j0 >= 2 && i0 + CW - 2 <= nx && j0 + CH - 2 <= ny;
    for (int t = threadIdx.x; t < CW * CH; t += NT) {
      const int cx = t % CW, cy = t / CW;
      int gi = i0 - 2 + cx, gj = j0 - 2 + cy;
      if (!interior) {
        gi = wrapi(gi, nx);
        gj = wrapi(gj, ny);
      }
      const size_t id = (size_t)gj * nx + gi;
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int k = 0; k < 4; ++k) W[(4 * f + k) * WPL + t] = __ldg(a.in.pt[f][k] + id);
    }
  }
  __syncthreads();

  // ---- phase 1: centre recovery of cells [i0-2, i0+TX+3) (Eq. center-node) ----
  // deviation form U_c = Ubar + 1/16 sum_corners (Ubar - U_V) + 1/4 sum_edges (Ubar - U_E)
  for (int t = threadIdx.x; t < (CW - 1) * (CH - 1); t += NT) {
    const int cx = t % (CW - 1), cy = t / (CW - 1);
    const int c = cy * CW + cx;
    const size_t id = (size_t)wrapi(j0 - 2 + cy, ny) * nx + wrapi(i0 - 2 + cx, nx);
    float ub[4], lo[4], sc[4] = {0.f, 0.f, 0.f, 0.f}, se[4] = {0.f, 0.f, 0.f, 0.f}, uc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ub[k] = __ldg(a.in.avg[k] + id);
      lo[k] = COMP ? __ldg(a.in.lo[k] + id) : 0.f;
    }
    auto node = [&](int fam, int idx) {
      Prim<float> w = {W[(4 * fam) * WPL + idx], W[(4 * fam + 1) * WPL + idx],
                       W[(4 * fam + 2) * WPL + idx], W[(4 * fam + 3) * WPL + idx]};
      return w;
    };
    const Prim<float> corners[4] = {node(0, c), node(0, c + 1), node(0, c + CW),
                                    node(0, c + CW + 1)};
    const Prim<float> edges[4] = {node(2, c), node(2, c + CW), node(1, c), node(1, c + 1)};
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      float u[4];
      cons_from_stored(corners[n], gas, u);
#pragma unroll
      for (int k = 0; k < 4; ++k) sc[k] += (ub[k] - u[k]) + lo[k];
      cons_from_stored(edges[n], gas, u);
#pragma unroll
      for (int k = 0; k < 4; ++k) se[k] += (ub[k] - u[k]) + lo[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) uc[k] = (ub[k] + lo[k]) + (0.0625f * sc[k] + 0.25f * se[k]);
    const Prim<float> w = stored_from_cons(uc, gas);
    if (!(gas.rho_ref + w.r > 0.f && gas.p_ref + w.p > 0.f)) bad |= FLAG_NONPHYSICAL;
    W[12 * WPL + c] = w.r;
    W[13 * WPL + c] = w.u;
    W[14 * WPL + c] = w.v;
    W[15 * WPL + c] = w.p;
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
      if (t < nV) {
        fam = 0; dx = t % (TX + 4); dy = t / (TX + 4);
      } else if (t < nV + nEv) {
        fam = 1; dx = (t - nV) % (TX + 4); dy = (t - nV) / (TX + 4);
      } else if (t < nV + nEv + nEh) {
        fam = 2; dx = (t - nV - nEv) % (TX + 3); dy = (t - nV - nEv) / (TX + 3);
      } else {
        fam = 3; dx = (t - nV - nEv - nEh) % (TX + 3); dy = (t - nV - nEv - nEh) / (TX + 3);
      }
      const int wc = (dy + 1) * CW + (dx + 1), dc = dy * DCW + dx;
      const float* Wf = W + 4 * fam * WPL;
      const float rk = gas.rho_ref + Wf[wc], uk = Wf[WPL + wc], vk = Wf[2 * WPL + wc];
      const float pkt = Wf[3 * WPL + wc], pk = gas.p_ref + pkt;
      if (!(rk > 0.f && pk > 0.f)) bad |= FLAG_NONPHYSICAL;
      const float c = sqrtf(gas.gamma * pk / rk);
      const float Z = rk * c, Zinv = 1.f / Z;
      const float r1 = c * dth;
      if (r1 > 0.5f) bad |= FLAG_CFL;
      float Gp[3][4], Guv[3][4];
      if (fam == 0) {
        LoadW<0, CW, WPL> ld = {W, wc};
        af_sac_V<float>(ld, pkt, uk, vk, Gp, Guv);
      } else if (fam == 1) {
        LoadW<1, CW, WPL> ld = {W, wc};
        af_sac_EV<float>(ld, pkt, uk, vk, Gp, Guv);
      } else if (fam == 2) {
        LoadW<2, CW, WPL> ld = {W, wc};
        af_sac_EH<float>(ld, pkt, uk, vk, Gp, Guv);
      } else {
        LoadW<3, CW, WPL> ld = {W, wc};
        af_sac_C<float>(ld, pkt, uk, vk, Gp, Guv);
      }
      float d[3];
      float* D0 = D + fam * 3 * DPL + dc;
      float* D1 = D + (4 + fam) * 3 * DPL + dc;
      increments_at(Gp, Guv, Z, Zinv, 0.5f * r1, d);
      D0[0] = d[0];
      D0[DPL] = d[1];
      D0[2 * DPL] = d[2];
      increments_at(Gp, Guv, Z, Zinv, r1, d);
      D1[0] = d[0];
      D1[DPL] = d[1];
      D1[2 * DPL] = d[2];
    }
  }
  __syncthreads();

  // ---- phase 3: point updates of cells [i0, i0+TX] x [j0, j0+TY] -------------
  // duration by duration; the points of duration s replace D(s) once every
  // thread is done reading it.
  constexpr int NPTS = G::NPTS;
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
      if (t >= NPTS) break;
      const int fam = t / PPL, rem = t - fam * PPL;
      const int px = rem % PW, py = rem / PW;
      const int ox = fam == 2 ? 1 : 0, oy = fam == 1 ? 1 : 0;
      const int wcP = (py + 2) * CW + (px + 2);  // W cell of the point's cell
      const float* Wf = W + 4 * fam * WPL;
      const float rp = Wf[wcP], up = Wf[WPL + wcP], vp = Wf[2 * WPL + wcP],
                  pp = Wf[3 * WPL + wcP];
      // first Picard stage from the point's own velocity (Eq. adv-footpoint)
      const float d1x = -th * up, d1y = -th * vp;
      if (!(fabsf(d1x) <= 1.f && fabsf(d1y) <= 1.f)) bad |= FLAG_REACH;
      float fx = 0.5f * ox + clamp1(d1x), fy = 0.5f * oy + clamp1(d1y);
      float flx = floorf(fx), fly = floorf(fy);
      float lx[3], ly[3];
      lagrange3(2.f * (fx - flx) - 1.f, lx);
      lagrange3(2.f * (fy - fly) - 1.f, ly);
      int c = wcP + (int)fly * CW + (int)flx;
      const float u1 = q2_eval<CW>(W + 1 * WPL, W + 5 * WPL, W + 9 * WPL, W + 13 * WPL, c, lx, ly);
      const float v1 = q2_eval<CW>(W + 2 * WPL, W + 6 * WPL, W + 10 * WPL, W + 14 * WPL, c, lx, ly);
      // the foot
      const float dfx = -th * u1, dfy = -th * v1;
      if (!(fabsf(dfx) <= 1.f && fabsf(dfy) <= 1.f)) bad |= FLAG_REACH;
      fx = 0.5f * ox + clamp1(dfx);
      fy = 0.5f * oy + clamp1(dfy);
      flx = floorf(fx);
      fly = floorf(fy);
      lagrange3(2.f * (fx - flx) - 1.f, lx);
      lagrange3(2.f * (fy - fly) - 1.f, ly);
      const int ix = (int)flx, iy = (int)fly;
      c = wcP + iy * CW + ix;
      Prim<float> wf;
      wf.r = q2_eval<CW>(W + 0 * WPL, W + 4 * WPL, W + 8 * WPL, W + 12 * WPL, c, lx, ly);
      wf.u = q2_eval<CW>(W + 1 * WPL, W + 5 * WPL, W + 9 * WPL, W + 13 * WPL, c, lx, ly);
      wf.v = q2_eval<CW>(W + 2 * WPL, W + 6 * WPL, W + 10 * WPL, W + 14 * WPL, c, lx, ly);
      wf.p = q2_eval<CW>(W + 3 * WPL, W + 7 * WPL, W + 11 * WPL, W + 15 * WPL, c, lx, ly);
      float d[3];
      Prim<float> nw;
      if (a.variant == 0) {
        // transported increment at the foot; rho from dp / c_f^2 (Sec. 6.1 step 4)
        const int dcf = (py + 1 + iy) * DCW + (px + 1 + ix);  // D cell of the foot cell
#pragma unroll
        for (int q = 0; q < 3; ++q)
          d[q] = q2_eval<DCW>(Ds + (0 * 3 + q) * DPL, Ds + (1 * 3 + q) * DPL,
                              Ds + (2 * 3 + q) * DPL, Ds + (3 * 3 + q) * DPL, dcf, lx, ly);
        const float rf = gas.rho_ref + wf.r, pf = gas.p_ref + wf.p;
        if (!(rf > 0.f && pf > 0.f)) bad |= FLAG_NONPHYSICAL;
        nw.r = wf.r + d[2] * rf / (gas.gamma * pf);
      } else {
        // additive update (Eq. barsukow-additive), acoustic rho closure at P
        const int dcp = (py + 1) * DCW + (px + 1);
#pragma unroll
        for (int q = 0; q < 3; ++q) d[q] = Ds[(fam * 3 + q) * DPL + dcp];
        nw.r = wf.r + d[2] * (gas.rho_ref + rp) / (gas.gamma * (gas.p_ref + pp));
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
    __syncthreads();  // D(s) is dead from here
    float* P = D + s * 12 * DPL;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int t = threadIdx.x + k * NT;
      if (t >= NPTS) break;
      const int fam = t / PPL, rem = t - fam * PPL;
      float* q = P + fam * 4 * PPL + rem;
      q[0] = res[k].x;
      q[PPL] = res[k].y;
      q[2 * PPL] = res[k].z;
      q[3 * PPL] = res[k].w;
    }
  }
  __syncthreads();

  // ---- phase 4: space-time Simpson fluxes (Sec. 3.1) and average update -------
  // vertical edges (i0+ex, j0+ey), ex in [0, TX], ey in [0, TY); horizontal edges
  // ex in [0, TX), ey in [0, TY].  Computed into registers, then stored over W.
  constexpr int NVE = G::NVE, NE = G::NE;
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
    const int fm = vert ? 1 : 2;              // E_v or E_h
    const int wa = (ey + 2) * CW + (ex + 2);  // W cell of V(ex, ey)
    const int wb = vert ? wa + CW : wa + 1;   // the edge's other vertex
    const int pa = ey * PW + ex, pb = vert ? pa + PW : pa + 1;
    float F[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      Prim<float> xa, xm, xb;
      if (s == 0) {
        xa = {W[0 * WPL + wa], W[1 * WPL + wa], W[2 * WPL + wa], W[3 * WPL + wa]};
        const float* Wm = W + 4 * fm * WPL;
        xm = {Wm[0 * WPL + wa], Wm[1 * WPL + wa], Wm[2 * WPL + wa], Wm[3 * WPL + wa]};
        xb = {W[0 * WPL + wb], W[1 * WPL + wb], W[2 * WPL + wb], W[3 * WPL + wb]};
      } else {
        const float* P = D + (s - 1) * 12 * DPL;
        xa = {P[0 * PPL + pa], P[1 * PPL + pa], P[2 * PPL + pa], P[3 * PPL + pa]};
        const float* Pm = P + fm * 4 * PPL;
        xm = {Pm[0 * PPL + pa], Pm[1 * PPL + pa], Pm[2 * PPL + pa], Pm[3 * PPL + pa]};
        xb = {P[0 * PPL + pb], P[1 * PPL + pb], P[2 * PPL + pb], P[3 * PPL + pb]};
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
      for (int q = 0; q < 4; ++q) F[q] = fmaf(wt, fa[q] + 4.f * fmid[q] + fb[q], F[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) flux[k][q] = lam * F[q];
  }
  __syncthreads();  // W is dead from here
#pragma unroll
  for (int k = 0; k < PERE; ++k) {
    const int t = threadIdx.x + k * NT;
    if (t >= NE) break;
#pragma unroll
    for (int q = 0; q < 4; ++q) FLX[q * NE + t] = flux[k][q];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < TX * TY; t += NT) {
    const int cx = t % TX, cy = t / TX;
    const int gi = i0 + cx, gj = j0 + cy;
    if (gi >= nx || gj >= ny) continue;
    const size_t id = (size_t)gj * nx + gi;
    const int fl = cy * PW + cx, fr = fl + 1;         // vertical edges x_i, x_{i+1}
    const int gb = NVE + cy * TX + cx, gt = gb + TX;  // horizontal edges y_j, y_{j+1}
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float* Fq = FLX + q * NE;
      if (COMP) {
        float hi = __ldg(a.in.avg[q] + id), lo = __ldg(a.in.lo[q] + id);
        comp_update(hi, lo, Fq[fl], Fq[fr], Fq[gb], Fq[gt]);
        a.out.avg[q][id] = hi;
        a.out.lo[q][id] = lo;
        if (!isfinite(hi)) bad |= FLAG_NONFINITE;
      } else {
        const float v = __ldg(a.in.avg[q] + id) - (Fq[fr] - Fq[fl]) - (Fq[gt] - Fq[gb]);
        a.out.avg[q][id] = v;
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
