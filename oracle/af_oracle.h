/*
 * af_oracle.h -- plain FP64 CPU oracle for one time step of the fully discrete
 * Active Flux method with transported acoustic increments (RB-TAI) and the
 * additive Roe-Barsukow (RB) point update, 2D Euler, periodic Cartesian grid.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this library; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA implementation.
 *
 * State layout (all functions): one contiguous block of 16*nx*ny doubles,
 * sixteen planes of nx*ny values, row-major (index j*nx+i):
 *   planes  0.. 3  cell averages  (rho, rho u, rho v, E)        of cell C_ij
 *   planes  4.. 7  vertex values  (rho, u, v, p) at (x_i,       y_j)
 *   planes  8..11  x-edge values  (rho, u, v, p) at (x_i,       y_{j+1/2})  [E_v]
 *   planes 12..15  y-edge values  (rho, u, v, p) at (x_{i+1/2}, y_j)        [E_h]
 * (Sec. 2, degrees of freedom and Fig. 1.)
 */
#ifndef AF_ORACLE_H
#define AF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_TAI 0
#define ORC_RB 1
#define ORC_FC 2 /* foot-centred exact acoustic update (Appendix C) */

/* error flags returned by orc_step (bitmask) */
#define ORC_FLAG_CFL 1          /* acoustic CFL c*dt/h > 1/2 at some node */
#define ORC_FLAG_NONPHYSICAL 2  /* rho <= 0 or p <= 0 where a sound speed is needed */
#define ORC_FLAG_NONFINITE 4    /* NaN/Inf in the new state */

/* node families used by the acoustic operator */
#define ORC_NODE_V 0
#define ORC_NODE_EV 1
#define ORC_NODE_EH 2
#define ORC_NODE_C 3

/* number of invariants written by orc_invariants */
#define ORC_NINV 12

/* One time step (Sec. 6.1, Algorithm) with the point update `variant`
 * (ORC_TAI, ORC_RB or ORC_FC).  in and out hold 16*nx*ny doubles each and must
 * not overlap.  Returns the OR of ORC_FLAG_* seen during the step; for ORC_FC
 * ORC_FLAG_CFL reports the compact footprint condition of Appendix C instead
 * of the nodal acoustic CFL. */
int orc_step(int nx, int ny, double h, double gamma, double dt, int variant,
             const double *in, double *out);

/* n_steps steps; returns OR of flags.  state is updated in place. */
int orc_run(int nx, int ny, double h, double gamma, double dt, int variant,
            int n_steps, double *state);

/* Centre recovery of every cell (Eq. center-node, Sec. 4 explicit indices):
 * wc holds 4*nx*ny doubles (rho, u, v, p planes).  Returns flags. */
int orc_center_recovery(int nx, int ny, double gamma, const double *state, double *wc);

/* Acoustic increments (Sec. 6.1, step 1) at every node of family `fam`
 * for duration tau: d holds 3*nx*ny doubles (du, dv, dp planes).
 * wc from orc_center_recovery. */
int orc_acoustic_increments(int nx, int ny, double h, double gamma, double tau, int fam,
                            const double *state, const double *wc, double *d);

/* Exact frozen acoustic operator at one node (Sec. 3.1; Appendix D block).
 * fam selects the wedge set; cells holds, for each adjacent cell in the
 * family's wedge order, 27 doubles: p[3][3], u[3][3], v[3][3] with index
 * [ix][iy] over the cell's Q2 nodes xi,eta in {-1,0,1}.
 * Wedge order -- V: NE, NW, SW, SE; E_v: right, left; E_h: upper, lower; C: full disk.
 * r = c_K tau / h, Z = rho_K c_K.  out = (p_ac, u_ac, v_ac). */
void orc_sac_node(int fam, const double *cells, double r, double Z, double *out);

/* Foot-centred exact frozen acoustic evolution (Appendix C) for the point of
 * family fam (V or an edge family) whose adjacent cells hold `cells` (layout
 * and order as in orc_sac_node), the disk of radius r = c_* tau / h centred at
 * the foot F = P + (fx, fy) h, frozen impedance Z = rho_* c_*.  Valid under the
 * compact footprint condition |fx| + r < 1/2, |fy| + r < 1/2.
 * out = (p, u, v) at F after the evolution. */
void orc_fc_node(int fam, const double *cells, double fx, double fy, double r, double Z,
                 double *out);

/* The 3x3 monomial block C^Theta_ab of Appendix D for wedge w
 * (0 NE,1 NW,2 SW,3 SE,4 right,5 left,6 upper,7 lower,8 full), ordered
 * (pi,u,v) x (pi,u,v), row-major into out[9]. */
void orc_sac_block(int w, int a, int b, double *out);

/* Primitive Q2 reconstruction R_h W at a point given in cell units
 * (X = (x-x_0)/h, Y = (y-y_0)/h); out = (rho,u,v,p).  wc from centre recovery. */
void orc_recon_eval(int nx, int ny, const double *state, const double *wc,
                    double X, double Y, double *out);

/* Global diagnostics in FP64 (see af_oracle.c for the list). */
void orc_invariants(int nx, int ny, double h, double gamma, const double *state,
                    double *out);

#ifdef __cplusplus
}
#endif
#endif
