/* Plain CPU oracle of one UGKWP time step (arXiv 2007.13091, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it; the
 * product (the ugkwp C-ABI library) never links, loads or calls it, and it
 * shares no code, header or constant with that library.
 *
 * Arrays of per-cell quantities are structure-of-arrays: component q of cell
 * i is at [q * n_cells + i].  Particle arrays are indexed by particle; vector
 * quantities are [component * n + k].
 */
#ifndef UGKWP_ORACLE_H
#define UGKWP_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_DIFFUSE_WALL = 1, ORC_BC_SPECULAR = 2, ORC_BC_INFLOW = 3, ORC_BC_OUTFLOW = 4 };
enum { ORC_FP64 = 0, ORC_MIXED = 1 };

typedef struct {
    int32_t type;      /* ORC_BC_* */
    int32_t pad_;
    double T_w;        /* wall temperature (diffuse wall) */
    double U_w[3];     /* wall velocity (diffuse wall), tangential */
    double W_in[5];    /* conservative state of the far field (inflow) */
} orc_bc;

typedef struct {
    double R, mu_ref, T_ref, omega, CFL, C2;
    double venkat_K;   /* Venkatakrishnan constant K: epsilon^2 = (K h)^3 (order 2) */
    double Pr;         /* Prandtl number of the wave's equilibrium heat flux (order 2):
                        * 0 or 1 = BGK as printed; otherwise the energy flux of the
                        * equilibrium part gains (1/Pr - 1) times its heat flux */
    int32_t order, N_ref, N_min, precision, max_crossings, n_bc;
    int32_t sampling;  /* 0: pairs U +/- sqrt(RT) X as printed; 1: the same pairs with X
                        * scaled per cell so that their thermal energy is exactly
                        * rho^hp |Omega| (3/2) R T (energy-matched sampling); 2: every
                        * particle drawn on its own from the first-order g_p
                        * (acceptance-rejection; order 2 only) */
    int32_t K;         /* internal degrees of freedom: rho E = rho |U|^2/2 + (3+K)/2 p; particles
                        * carry an internal energy e ~ R T chi^2_K (0 <= K <= 8; K > 0 with
                        * sampling 0 only) */
    uint64_t seed;
    orc_bc bc[16];
} orc_params;

typedef struct orc_sim orc_sim;

/* ---- elementary pins ---------------------------------------------------- */
/* which: 0 exp_d, 1 log_d, 2 sin(2 pi x), 3 cos(2 pi x) */
void orc_math_d(int which, const double* x, double* y, int64_t n);
void orc_math_logf(const float* x, float* y, int64_t n);
/* sin(2 pi x), cos(2 pi x) in binary32 (the particle arithmetic of the mixed mode) */
void orc_math_sincos2pi_f(const float* x, float* s, float* c, int64_t n);
void orc_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
void orc_philox32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* q1..q5, then the two free-transport coefficients of the collisional wave:
 * a4 = q4 - dt e^{-dt/tau}, a5 = q5 + dt^2/2 e^{-dt/tau}. */
void orc_qcoef(double dt, double tau, double q[7]);
/* Moments of a unit-density Maxwellian (U, lambda) with K = 0, normal n:
 * H[5] = int_{half} g psi du, G[5] = int_{half} u.n g psi du,
 * half = +1 (u.n > 0), -1 (u.n < 0) or 0 (all u). */
void orc_maxwell_moments(const double U[3], double lam, const double n[3], int half, int32_t K,
                         double H[5], double G[5]);
/* Time-integrated wave flux of one face (F^eq + F^{fr,wave}, per unit area,
 * normal from L to R).  kind: 0 interior, or an ORC_BC_* type with the ghost
 * built from WL (and bc).  rhoh = hydrodynamic density rho^h of each side.
 * gks != 0: the flux of a step without particles (free transport q4). */
int orc_face_flux(const orc_params* p, int kind, const double WL[5], double rhohL,
                  const double WR[5], double rhohR, const double n[3], double dt,
                  double tau_wall, const orc_bc* bc, int32_t gks, double F[5]);

/* ---- simulation --------------------------------------------------------- */
orc_sim* orc_create(const orc_params* p, int32_t n_nodes, const double* xyz,
                    int32_t n_tets, const int32_t* tets, int32_t n_bfaces,
                    const int32_t* bfaces, const int32_t* btags, const double* W0,
                    char* err, int32_t errlen);
void orc_free(orc_sim* s);
int orc_step(orc_sim* s, char* err, int32_t errlen);
/* One step of the gas-kinetic scheme (no particles; the state must hold none):
 * global time step (local = 0) or local time steps (local = 1). */
int orc_gks_step(orc_sim* s, int32_t local, char* err, int32_t errlen);

/* sizes: [n_cells, n_faces, n_boundary_faces, n_particles, step] */
void orc_sizes(const orc_sim* s, int64_t out[5]);
/* Geometry (which): 0 vol[nc], 1 centroid[3][nc], 2 face normal[3][nf],
 * 3 face area[nf], 4 face owner (as double)[nf], 5 face neighbour (-1 boundary)[nf],
 * 6 dS[3][nc], 7 face plane offset d[nf] */
int orc_geometry(const orc_sim* s, int which, double* out);
/* State export.  Any pointer may be NULL.  scal = [step, e_0..e_4] (int64),
 * t = simulation time, e = the particles' internal energies (0 when K = 0). */
void orc_get_state(const orc_sim* s, double* W, uint64_t* id, int32_t* cell,
                   double* x, double* u, double* m, int64_t* scal, double* t, double* e);
/* State import (teacher forcing).  Positions/velocities (and internal
 * energies, read when K > 0; e may be NULL) must be exactly representable in
 * the particle precision. */
int orc_set_state(orc_sim* s, const double* W, int64_t n, const uint64_t* id,
                  const int32_t* cell, const double* x, const double* u, const double* m,
                  const int64_t* scal, double t, const double* e, char* err, int32_t errlen);
/* Diagnostics of the last step (which):
 *  0 dt (1 value), 1 tau[nc], 2 rho_h[nc] (before sampling), 3 n_sam[nc],
 *  4 m_sam[nc], 5 wave flux F[5][nf], 6 particle flux F^{fr,p}[5][nc] (fixed point,
 *  int64 written as raw 8 bytes), 7 survivor mass sum[nc] (int64 raw),
 *  8 survivor count[nc], 9 counters [n_tracked, n_collided, n_exited, n_lost,
 *  n_crossings, n_wall_hits, n_sampled] */
int orc_last(const orc_sim* s, int which, void* out);

/* Cell preparation of the current state without stepping: primitives, tau,
 * rho^h, dt and the sampling counts (then readable with orc_last 0..4). */
int orc_prepare(orc_sim* s, char* err, int32_t errlen);
/* The particles cell `cell` samples at the current step (after orc_prepare):
 * returns their number n and fills up to cap of them (x, u as [k][3]). */
int64_t orc_sample_cell(const orc_sim* s, int32_t cell, int64_t cap, uint64_t* id, double* x, double* u, double* m,
                        double* e);
/* First-order g_p sampling (sampling = 2), after orc_prepare: the cell's
 * acceptance polynomial phi(X) = a0 + L.X + X^T Q X + (C.X)|X|^2 of X = (u - U)
 * / sqrt(RT) and its bound: [a0, L(3), Qxx, Qyy, Qzz, Qxy, Qxz, Qyz, C(3), M].
 * -1 if the state has none. */
int orc_gp_coefficients(const orc_sim* s, int32_t cell, double out[14]);
/* n acceptance-rejection draws X[n][3] of first-order g_p for the given
 * coefficients, particle ids id0 .. id0 + n - 1 at `step`, in the particle
 * precision (ORC_FP64 / ORC_MIXED). */
void orc_gp_draw(int32_t precision, uint64_t seed, uint64_t step, const double coef[14], uint64_t id0, int64_t n,
                 double* X);

/* Second-order pieces (order 2).  Gradients of the current state [5][3][nc]
 * and [3][nc] (limited or not).  Slope moment int u_n u_d (a.psi) psi g du of
 * a unit-density Maxwellian in a face frame (u along the normal; U given in
 * that frame; half = +1, -1, 0).  Micro slope a with <psi psi^T> a = b.
 * Second-order flux of one interior face from cell states, limited gradients
 * ([q][d] row-major) and centroid-to-face vectors. */
int orc_gradients(orc_sim* s, int limited, double* gradW, double* gradH);
void orc_slope_moment(const double U[3], double lam, int half, int32_t K, const double a[5], int d, double out[5]);
void orc_micro_slope(const double U[3], double lam, int32_t K, const double b[5], double a[5]);
int orc_face_flux_o2(const orc_params* p, const double WL[5], double rhohL, const double gWL[15], const double gHL[3],
                     const double dxL[3], const double WR[5], double rhohR, const double gWR[15],
                     const double gHR[3], const double dxR[3], const double n[3], double dt, int32_t gks,
                     double F[5]);

/* Frozen-particle wave map (first order only): K steps of
 *   W^{n+1} = W^n - sum_f (+/-) F_f(W^n; theta) |S_f| / |Omega| + pf^n / |Omega|
 * from W0 [5][nc] with the recorded dt[K], particle densities rho_p[K][nc]
 * (rho^h = rho - rho^p) and particle fluxes pflux[K][5][nc] (scaled, per cell).
 * theta = (rho_inf, U_inf, T_w) sets every far-field state equal to the first
 * one (density, speed along its direction, same temperature) and the
 * temperature of the diffuse walls with a listed tag.  J = sum over steps and
 * listed boundary faces of F[c] |S|, c = 1 (functional 0, drag) or 4
 * (functional 1, wall heat flux).  orc_frozen_objective: out = [J, dJ/dtheta]
 * by forward-mode dual numbers; orc_frozen_value: J alone in binary64.
 * Return 0, or -1 (order != 1, K < 1, unknown functional). */
int orc_frozen_objective(const orc_sim* s, int32_t K, const double* W0, const double* dt, const double* rho_p,
                         const double* pflux, const double theta[3], int32_t functional, const int32_t* tags,
                         int32_t n_tags, double out[4]);
int orc_frozen_value(const orc_sim* s, int32_t K, const double* W0, const double* dt, const double* rho_p,
                     const double* pflux, const double theta[3], int32_t functional, const int32_t* tags,
                     int32_t n_tags, double* J);

/* The same map at second order (the simulation's order must be 2): limited
 * least-squares reconstruction at interior faces, first-order boundary faces,
 * far-field ghosts at theta, binary64 only.  phi [K][6][nc] holds the limiter
 * values of W (5) and rho^h: computed and written with record != 0, read
 * otherwise (the limiter frozen).  Return 0, or -1 (order != 2, K != 0 internal
 * degrees of freedom, K < 1, unknown functional). */
int orc_frozen_o2_value(const orc_sim* s, int32_t K, const double* W0, const double* dt, const double* rho_p,
                        const double* pflux, const double theta[3], int32_t functional, const int32_t* tags,
                        int32_t n_tags, double* phi, int32_t record, double* J);

/* Track one particle with the simulation's mesh and parameters (sampled checks
 * at sizes where a whole oracle step would be slow).  io_x/io_u are [3];
 * the particle precision follows the simulation.  Returns the status bits
 * 1 collided, 2 exited, 4 lost; *cell_out the end tet; *ncross the crossings. */
int orc_track_one(const orc_sim* s, uint64_t id, int32_t cell, double* io_x, double* io_u, double* io_e,
                  double tau_cell, double dt, int64_t step, int32_t* cell_out, int32_t* ncross);

#ifdef __cplusplus
}
#endif
#endif
