/*
 * ugkwp.h -- C-ABI of the GB300 (sm_103a) unified gas-kinetic wave-particle
 * (UGKWP) time step on unstructured tetrahedral meshes.
 *
 * The method is that of Chen, Zhu & Xu, "A three-dimensional unified
 * gas-kinetic wave-particle solver for flow computation in all regimes"
 * (arXiv 2007.13091), Sec. 2: the cell-averaged conservative variables
 * W = (rho, rho U, rho E) evolve by the finite-volume law of Eq. (FVmacroEq)
 * with the multiscale flux of Sec. 2.1 (equilibrium part F^eq and the
 * free-transport part of the collisional hydrodynamic wave, Sec. 2.3), while
 * the collisionless part of the gas is carried by simulation particles
 * (Sec. 2.2) whose free-transport time t_f = min(-tau ln eta, dt) decides
 * whether they survive the step; particles are streamed through the tets,
 * counted into the particle flux F^{fr,p}, removed when collisional, and the
 * collisionless fraction e^{-dt/tau} of the hydrodynamic wave is re-sampled as
 * particles at the start of every step (Sec. 2.4 (b)).
 *
 * Conventions for every entry point:
 *  - All functions return 0 (UGKWP_OK) or a negative UGKWP_E_* status; the
 *    message of the last failure in the calling thread is available through
 *    ugkwp_last_error().  Invalid arguments are reported synchronously.
 *  - Device-side failures (capacity, lost particles, fixed-point overflow,
 *    non-physical states) set a device error word; it is read and returned by
 *    the next call that synchronises (ugkwp_step with stats, ugkwp_moments,
 *    ugkwp_export_state, ugkwp_sync).  No call traps or hangs the GPU: every
 *    data-dependent device loop has an iteration cap.
 *  - Per-cell arrays are structure-of-arrays, component-major: component q of
 *    cell i is at [q * n_cells + i].  Per-particle vectors are [3][n].
 *  - Objects are opaque; calls on one object are not thread-safe.
 *  - The library allocates no device memory: the caller provides one
 *    workspace (size from ugkwp_query_sizes) that must outlive the simulation.
 */
#ifndef UGKWP_H
#define UGKWP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
    UGKWP_OK = 0,
    UGKWP_E_ARG = -1,            /* invalid argument */
    UGKWP_E_MESH = -2,           /* invalid mesh (inverted tet, unmatched face, ...) */
    UGKWP_E_CUDA = -3,           /* CUDA runtime error */
    UGKWP_E_WORKSPACE = -4,      /* workspace missing, too small or misaligned */
    UGKWP_E_CAPACITY = -5,       /* particle capacity exceeded (step aborted its writes) */
    UGKWP_E_TRACK_LIMIT = -7,    /* a particle exceeded max_crossings face crossings */
    UGKWP_E_FIXED_OVERFLOW = -8, /* a particle's fixed-point flux left the int64 range */
    UGKWP_E_NONFINITE = -9,      /* non-positive density/pressure or non-finite state */
    UGKWP_E_STATE = -10,         /* call out of order / inconsistent imported state */
    UGKWP_E_UNSUPPORTED = -11    /* feature not available in this build */
};

/* ------------------------------------------------------ boundary types
 * Sec. 2.4 (e) gives the diffuse isothermal wall; the paper's test cases also
 * use far-field and symmetry (specular) boundaries. */
enum {
    UGKWP_BC_DIFFUSE_WALL = 1, /* isothermal wall (T_w, U_w): wave re-emitted as g_w,
                                  particles re-emitted diffusely, full accommodation */
    UGKWP_BC_SPECULAR = 2,     /* symmetry plane: mirror ghost, specular particles */
    UGKWP_BC_FARFIELD = 3,     /* prescribed far-field/inflow Maxwellian W_in: all-hydro
                                  ghost, particles leaving the domain are absorbed */
    UGKWP_BC_OUTFLOW = 4       /* zero-gradient ghost (ghost = interior), absorbing */
};

/* Particle precision.  FP64: particle state and tracking in binary64.
 * MIXED: particle position, velocity, t_f and tracking in binary32; particle
 * mass, fluxes (fixed point), relaxation times and all cell/face arithmetic
 * stay binary64. */
enum { UGKWP_FP64 = 0, UGKWP_MIXED = 1 };
enum { UGKWP_SAMPLE_MAXWELL = 0, UGKWP_SAMPLE_ENERGY_MATCHED = 1, UGKWP_SAMPLE_GP1 = 2 };

/* Which quantity ugkwp_moments returns (all [5][n_cells] unless stated). */
enum {
    UGKWP_W = 0,     /* conservative W = (rho, rho U, rho E) of the whole gas */
    UGKWP_WP = 1,    /* W^p: conservative variables carried by the particles (Eq. W^p) */
    UGKWP_WH = 2,    /* W^h = W - W^p, the hydrodynamic wave */
    UGKWP_PRIM = 3,  /* primitives (rho, U_x, U_y, U_z, T) of W */
    UGKWP_WBAR = 4   /* time average W-bar = sum dt^n W^n / sum dt^n (Sec. 2.4 (c)), see ugkwp_average */
};

/* ------------------------------------------------------------------ types */
typedef struct ugkwp_mesh ugkwp_mesh;
typedef struct ugkwp_sim ugkwp_sim;

/* Mesh description.  All arrays are host memory owned by the caller and are
 * copied by ugkwp_mesh_load.  Every tet must have positive volume with its
 * nodes in the given order; every face must be shared by two tets or listed
 * once in bfaces with a tag in [0, n_bc). */
typedef struct {
    int32_t n_nodes;
    int32_t n_tets;              /* < 2^24 (particle ids hold the birth cell in 24 bits) */
    int32_t n_bfaces;
    int32_t reserved;
    const double* xyz;           /* [n_nodes][3] node coordinates */
    const int32_t* tets;         /* [n_tets][4] node indices */
    const int32_t* bfaces;       /* [n_bfaces][3] node indices of boundary faces */
    const int32_t* bface_tags;   /* [n_bfaces] index into ugkwp_params.bc */
} ugkwp_mesh_desc;

typedef struct {
    int32_t type;                /* UGKWP_BC_* */
    int32_t reserved;
    double T_w;                  /* diffuse wall temperature */
    double U_w[3];               /* diffuse wall velocity (tangential to the wall) */
    double W_in[5];              /* far-field conservative state */
} ugkwp_bc;

/* Gas and scheme parameters.  tau = mu_ref/p (T/T_ref)^omega (Sec. 2, Eq.
 * tau_via_T_ref); dt = CFL min_i |Omega_i| / sum_d Lambda_i^d (Sec. 2.4 (a));
 * face relaxation time adds C2 |p_l - p_r|/|p_l + p_r| dt (Sec. 2.4 (d));
 * N_ref, N_min control the sampling (Sec. 2.4 (b)). */
typedef struct {
    double R;                    /* specific gas constant */
    double mu_ref, T_ref, omega; /* viscosity law */
    double Pr;                   /* Prandtl number (0 or 1: BGK).  Otherwise, at order 2, the
                                  * energy flux of the wave's equilibrium part gains (1/Pr - 1)
                                  * times its heat flux relative to the face velocity (the
                                  * GKS Prandtl fix; particles stay BGK).  E_ARG if < 0 or
                                  * not finite */
    double CFL;                  /* Courant number C in (0, 1] */
    double C2;                   /* numerical-dissipation constant (>= 0) */
    double venkat_K;             /* Venkatakrishnan constant K (>= 0): epsilon^2 = (K |Omega|^(1/3))^3 */
    int32_t order;               /* reconstruction order: 1, or 2 (least-squares gradients with
                                  * Venkatakrishnan's limiter at interior faces, Sec. 2.1) */
    int32_t N_ref;               /* reference particle number per cell (> 0) */
    int32_t N_min;               /* minimum particles per cell after sampling (>= 0) */
    int32_t precision;           /* UGKWP_FP64 or UGKWP_MIXED */
    int32_t max_crossings;       /* cap on face crossings per particle and step (> 0) */
    int32_t n_bc;                /* number of used entries of bc (<= 16) */
    int32_t sampling;            /* UGKWP_SAMPLE_MAXWELL: pairs U +/- sqrt(RT) X (Sec. 2.4 (b));
                                  * UGKWP_SAMPLE_ENERGY_MATCHED: the same pairs with X scaled per
                                  * cell so that their thermal energy is exactly
                                  * rho^hp |Omega| (3/2) R T (a variance reduction);
                                  * UGKWP_SAMPLE_GP1: every particle drawn on its own from the
                                  * first-order g_p of Sec. 2.2, g - c (u.grad g + g_t) with
                                  * c = tau - dt e^{-dt/tau}/(1 - e^{-dt/tau}), by
                                  * acceptance-rejection (order 2 only: the cell slopes) */
    int32_t K;                   /* internal degrees of freedom (Sec. 2.2): rho E = rho |U|^2/2 +
                                  * (3+K)/2 p, and each particle carries an internal energy e
                                  * (phi = m (1, u, (|u|^2 + e)/2)) sampled as R T chi^2_K and
                                  * re-drawn at diffuse walls from T_w.  0 <= K <= 8; K > 0 needs
                                  * UGKWP_SAMPLE_MAXWELL; the adjoint needs K = 0 */
    uint64_t seed;               /* Philox4x64-10 key word 0 */
    int64_t particle_capacity;   /* particles the device buffers hold (< 2^31) */
    ugkwp_bc bc[16];
} ugkwp_params;

typedef struct {
    size_t workspace_bytes;      /* device bytes the caller must provide */
    int64_t n_cells, n_faces, n_bfaces;
} ugkwp_sizes;

/* Step statistics (filled when requested; forces a stream synchronisation). */
typedef struct {
    double t, dt;                /* time after the last step, its time step */
    int64_t step;                /* steps taken so far */
    int64_t n_particles;         /* particles alive after the last step */
    int64_t n_tracked;           /* particles moved in the last step (old + sampled) */
    int64_t n_sampled, n_collided, n_exited, n_lost, n_crossings, n_wall_hits;
    int64_t n_moves_total;       /* particle moves summed over every step since init */
    int64_t n_movers;            /* particles of the last step whose counting flux is not zero (they
                                  * left their start cell, met a wall or left the domain) */
} ugkwp_stats;

/* Host-side image of the simulation state for checkpoint/restart and for
 * teacher-forced comparison.  All pointers are caller-owned host buffers:
 * W [5][n_cells]; id, cell, m, e [n]; x, u [3][n] (binary64; in MIXED mode
 * the values are binary32 numbers widened exactly).  e: the internal energies
 * (read and written when K > 0; may be NULL when K = 0).  exps are the base-2
 * exponents of the fixed-point quanta of (mass, 3 x momentum, energy). */
typedef struct {
    int64_t n_particles;
    int64_t step;
    double t;
    int32_t exps[5];
    int32_t reserved;
    double* W;
    uint64_t* id;
    int32_t* cell;
    double* x;
    double* u;
    double* m;
    double* e;
} ugkwp_state;

/* ---------------------------------------------------------------- mesh */

/* Build the mesh object: validates the tets (positive volume), matches faces
 * on sorted node triples, assigns boundary tags and precomputes geometry
 * (unit face normals from owner to neighbour, areas, plane offsets, volumes,
 * the projected areas Delta S of Sec. 2.4 (a)).  Host only; no GPU needed.
 * Errors: UGKWP_E_ARG (NULL/size), UGKWP_E_MESH (with a message). */
int ugkwp_mesh_load(const ugkwp_mesh_desc* d, ugkwp_mesh** out);
int ugkwp_mesh_free(ugkwp_mesh* m);

/* Device workspace needed for (mesh, params).  Host only. */
int ugkwp_query_sizes(const ugkwp_mesh* m, const ugkwp_params* p, ugkwp_sizes* out);

/* Create a simulation: copies the mesh geometry and the initial state W0
 * (host, [5][n_cells], conservative) into the caller's device workspace
 * (>= workspace_bytes, 256-byte aligned, owned by the caller and used until
 * ugkwp_free), and binds the CUDA stream (cudaStream_t, NULL = legacy default)
 * on which every later call enqueues its work (a stream of its own lets each
 * step's wave and particle kernels overlap as designed; on the legacy default
 * stream the replayed steps ran up to 30% slower).  No particles exist yet: the
 * first step samples e^{-dt/tau} of every cell as particles.  The mesh object
 * may be freed afterwards.  Errors: UGKWP_E_ARG, UGKWP_E_WORKSPACE,
 * UGKWP_E_NONFINITE (W0 with rho <= 0 or p <= 0), UGKWP_E_CUDA. */
int ugkwp_init(const ugkwp_mesh* m, const ugkwp_params* p, const double* W0,
               void* d_workspace, size_t workspace_bytes, void* cuda_stream,
               ugkwp_sim** out);
int ugkwp_free(ugkwp_sim* s);

/* Advance n_steps time steps (Sec. 2.2 procedure, Eq. update_macro_variables),
 * asynchronously on the bound stream.  Within each step the wave flux runs on
 * a second, library-owned stream forked from and joined back into the bound
 * stream, so the caller sees one stream-ordered step.  If st is non-NULL the
 * call waits for the stream, fills st and returns any device-side error. */
int ugkwp_step(ugkwp_sim* s, int32_t n_steps, ugkwp_stats* st);

/* Wait for the stream and return (then clear) any device-side error. */
int ugkwp_sync(ugkwp_sim* s);

/* Start-up steps of the gas-kinetic scheme (GKS), the method without
 * particles (Sec. 3.2), for the initial field of a steady case (Sec. 4.3, 4.4: GKS
 * start-up, with local time stepping): per step, no particle is sampled
 * (W^h = W) and the wave flux carries the whole free transport (q4, q5 in
 * place of a4, a5).  local_dt = 0: the global time step; t advances.
 * local_dt = 1: local time steps dt_i = CFL |Omega_i| / sum_d Lambda_i^d, each
 * face integrated over the smaller dt of its cells (the interior cell's at a
 * boundary) and cell i advanced by dt_i times the mean flux rates (a pseudo
 * time: t stays).  Neither advances the step counter or the time averages.
 * Asynchronous like ugkwp_step (st, if non-NULL, gets t and dt and syncs);
 * the call itself reads the particle count first (synchronising).
 * Errors: E_ARG, E_STATE (the state holds particles: GKS steps come before
 * the first ugkwp_step), E_NONFINITE at the next synchronising call. */
int ugkwp_gks_steps(ugkwp_sim* s, int32_t n_steps, int32_t local_dt, ugkwp_stats* st);

/* Time averaging for steady states (Sec. 2.4 (c)).  start != 0 resets the
 * sums and, from the next step on, adds dt^n W^n (the state after step n) to
 * them; start == 0 stops adding (the sums stay readable).  UGKWP_WBAR then
 * returns sum dt^n W^n / sum dt^n; *t_avg (may be NULL) receives sum dt^n.
 * E_STATE for UGKWP_WBAR before any averaged step. */
int ugkwp_average(ugkwp_sim* s, int32_t start);
int ugkwp_average_time(ugkwp_sim* s, double* t_avg);

/* Gradient-length local Knudsen number Kn_GLL = l |grad rho| / rho per cell
 * (the diagnostic the paper plots), with the unlimited least-squares gradient
 * of rho over the 4 face neighbours (boundary ghosts as in the reconstruction)
 * and the VHS mean free path l = 2 (5 - 2 omega)(7 - 2 omega) / 15
 * mu / (rho sqrt(2 pi R T)), mu = mu_ref (T / T_ref)^omega.  out: host
 * [n_cells] (synchronising). */
int ugkwp_kn_gll(ugkwp_sim* s, double* out);

/* Copy a per-cell quantity (UGKWP_W, _WP, _WH, _PRIM, _WBAR) to out: a device
 * pointer (out_on_device = 1, enqueued on the stream) or host memory
 * (out_on_device = 0, synchronising).  [5][n_cells] doubles. */
int ugkwp_moments(ugkwp_sim* s, int32_t which, double* out, int32_t out_on_device);

/* State image: ugkwp_state_info fills the scalar fields (n_particles, step,
 * t, exps); ugkwp_export_state also fills the arrays (which must hold
 * n_particles entries).  ugkwp_import_state replaces the simulation state
 * (W, particles, step, t, exps) from host arrays.  Synchronising.  The
 * arrays are copied to the device as they are and every particle is checked
 * and converted to the particle precision there, into the simulation's spare
 * particle buffer, before its state changes: a rejected image leaves the
 * simulation as it was.  In mixed precision the binary64 positions,
 * velocities and internal energies pass through a device staging buffer
 * (3 n_cells + 6 n_particles doubles, 7 n_particles with K > 0) allocated by
 * the call, kept between imports and freed with ugkwp_free; the native image
 * below needs none.  Host arrays in page-locked memory copy fastest.
 * Errors: UGKWP_E_ARG, UGKWP_E_CAPACITY, UGKWP_E_STATE (particle outside the
 * mesh index range or not representable in the particle precision). */
int ugkwp_state_info(ugkwp_sim* s, ugkwp_state* st);
int ugkwp_export_state(ugkwp_sim* s, ugkwp_state* st);
int ugkwp_import_state(ugkwp_sim* s, const ugkwp_state* st);

/* Native image of the simulation state, for checkpoint and restart of the
 * same mesh and precision: the particles as the simulation stores them, so
 * that no conversion is needed either way.  Like ugkwp_state, except that x,
 * u and e hold real_size bytes per value (4 in MIXED, 8 in FP64; set by the
 * export, checked by the import): in MIXED x is the binary32 offset of the
 * particle from the anchor of its tet (a point of the tet fixed by
 * ugkwp_init: the position is anchor + offset, exactly, in binary64), u and e
 * the binary32 velocity and internal energy; in FP64 the binary64 values.
 * e may be NULL when K = 0 (the export then writes zeros into it if given).
 * The export holds the live particles in buffer order (the arrays must hold
 * n_particles entries; with n_particles too small it reports UGKWP_E_ARG and
 * fills only the scalar fields).  The import copies the arrays as they are
 * into the simulation's spare particle buffer and checks there every
 * particle's cell (in [0, n_cells)) and internal energy (>= 0) before the
 * state changes; a rejected image leaves the simulation as it was.
 * Synchronising.  Errors: UGKWP_E_ARG (NULL argument, real_size of another
 * precision, e missing with K > 0), UGKWP_E_CAPACITY, UGKWP_E_STATE. */
typedef struct {
    int64_t n_particles;
    int64_t step;
    double t;
    int32_t exps[5];
    int32_t real_size;
    double* W;
    uint64_t* id;
    int32_t* cell;
    void* x;
    void* u;
    double* m;
    void* e;
} ugkwp_state_native;
int ugkwp_export_state_native(ugkwp_sim* s, ugkwp_state_native* st);
int ugkwp_import_state_native(ugkwp_sim* s, const ugkwp_state_native* st);

/* Diagnostics of the last step, copied to host memory (synchronising):
 *  0 dt (1 double), 1 tau [n_cells], 2 rho^h before sampling [n_cells],
 *  3 N_sam [n_cells] (int64), 4 m_sam [n_cells], 5 wave flux
 *  F^eq + F^{fr,wave} per unit area [5][n_faces] (face numbering: by owner
 *  tet then its local face; after a GKS step with local time steps the mean
 *  rate F / dt_f), 6 particle flux F^{fr,p} in fixed point
 *  [5][n_cells] (int64), 7 survivor mass in fixed point [n_cells] (int64),
 *  8 survivor count [n_cells] (int64); at order 2 only: 9 limited gradients
 *  of W [5][3][n_cells] (component, direction, cell), 10 limited gradient of
 *  rho^h [3][n_cells]. */
int ugkwp_last(ugkwp_sim* s, int32_t which, void* host_out);

/* Kernel classes of one step, in launch order (for ugkwp_timing_read). */
enum {
    UGKWP_K_RESET = 0, UGKWP_K_CELL_PREP, UGKWP_K_SAMPLE_COUNT, UGKWP_K_SCAN,
    UGKWP_K_SCATTER, /* no kernel launches in this class: the tracking kernel compacts the survivors */
    UGKWP_K_SAMPLE, UGKWP_K_TRACK, UGKWP_K_FLUX, UGKWP_K_UPDATE, UGKWP_K_MOVERS, UGKWP_K_GRADIENTS,
    UGKWP_K_FLUX_O2, UGKWP_N_KERNELS
};

/* ---- launch configuration and autotuning -------------------------------
 * Grid sizes and block shapes of the step kernels that loop over their work.
 * Results do not depend on them (every particle draws from its own
 * counter-based stream and every sum over particles is fixed point), only the
 * speed does. */
typedef struct {
    int32_t particle_blocks;     /* blocks of the sampling, tracking and movers kernels (> 0) */
    int32_t wave_blocks;         /* blocks of the persistent second-order wave kernels (> 0) */
    int32_t track_threads;       /* particles per tracking tile, one per thread of a block: 128 or 256 */
    int32_t smem_carveout;       /* preferred shared-memory carveout of the step's kernels, percent of
                                  * the largest (0..100), or -1 for the driver's choice (default 58).
                                  * A kernel attribute: it holds for every simulation of the process */
} ugkwp_launch_cfg;

int ugkwp_get_launch_cfg(const ugkwp_sim* s, ugkwp_launch_cfg* out);
/* Takes effect at the next step (the step graphs are recaptured). */
int ugkwp_set_launch_cfg(ugkwp_sim* s, const ugkwp_launch_cfg* cfg);
/* Autotuner: two stages of trials, each trial 2 warm-up steps and
 * steps_per_trial timed steps (even, >= 2) on the bound stream: (1) tracking
 * block of 128 or 256 threads x carveout (the driver's choice, or 58% for every
 * kernel of the step) at 1024 resident tracking threads per SM and one wave
 * block per SM; (2) for the fastest, 512, 1024 or 2048 resident tracking threads
 * per SM (the grid split in its two launches) x 1 or 2 wave blocks per SM (order
 * 2).  Keeps the fastest and returns it in *best (may be NULL).  The trial
 * steps advance the simulation like any other steps.  E_STATE while per-kernel
 * timing is on. */
int ugkwp_autotune(ugkwp_sim* s, int32_t steps_per_trial, ugkwp_launch_cfg* best);

/* ---- batches of independent simulations --------------------------------
 * A batch steps n simulations of any sizes and parameters together: every
 * step pair of all members is captured into one CUDA graph in which the
 * members run concurrently on the batch's own streams, and the graph is
 * launched on cuda_stream (NULL: the legacy default stream).  Each member
 * keeps its own state, random streams and results, bit for bit the same as
 * when stepped alone.  Members must be distinct; while stepped through a batch
 * a member is read or stepped on its own only after ugkwp_batch_sync.  The
 * batch does not own its members (free it before them). */
typedef struct ugkwp_batch ugkwp_batch;

int ugkwp_batch_create(ugkwp_sim* const* sims, int32_t n_sims, void* cuda_stream, ugkwp_batch** out);
/* Enqueue n_steps steps of every member (asynchronous on cuda_stream). */
int ugkwp_batch_step(ugkwp_batch* b, int32_t n_steps);
/* Wait for the batch's stream; returns the first member's device-side error
 * (the message names the member index). */
int ugkwp_batch_sync(ugkwp_batch* b);
/* The autotuner over the whole batch: one grid pair for all members, chosen by
 * the time of batch step pairs (trial steps advance every member). */
int ugkwp_batch_autotune(ugkwp_batch* b, int32_t steps_per_trial, ugkwp_launch_cfg* best);
int ugkwp_batch_free(ugkwp_batch* b);

/* Per-kernel timing with CUDA events recorded on the bound stream around each
 * kernel launch of ugkwp_step while enabled (enable != 0).  ugkwp_timing_read
 * synchronises and returns, per kernel class, the summed device time in
 * milliseconds (ms[UGKWP_N_KERNELS]) of the launches timed since the last
 * read, and the number of kernels launched since ugkwp_init
 * (launches[UGKWP_N_KERNELS], counted whether or not timing is enabled; the
 * scan class counts its two kernels); at order 2 the flux class times the
 * boundary faces and UGKWP_K_FLUX_O2 the interior faces; either pointer may
 * be NULL.  The timed
 * sums are reset by the read. */
int ugkwp_timing_enable(ugkwp_sim* s, int32_t enable);
int ugkwp_timing_read(ugkwp_sim* s, double* ms, int64_t* launches);

/* ---- adjoint of the wave update with the particle sample frozen ---------
 * The call takes n_steps = K real steps of the simulation (advancing it like
 * ugkwp_step), recording each step's time step, particle density rho^p and
 * particle flux F^{fr,p}.  With those frozen, the wave part of the K steps
 * from the state at the call is a smooth map
 *   W^{n+1} = W^n - sum_f (+/-) F_f(W^n; theta) |S_f| / |Omega| + F^{fr,p,n} / |Omega|
 * (the step's flux of Sec. 2.1, 2.3, 2.4 (d), (e): first order, or at order 2
 * the limited least-squares reconstruction at interior faces, boundary faces
 * first order), and
 *   J = sum_n sum_{boundary faces with a tag in wall_tags} F_f[c] |S_f|
 * with c = 1 for functional 0 (x momentum delivered to the walls: drag) and
 * c = 4 for functional 1 (energy: wall heat flux), wave part only.
 * theta = (rho_inf, U_inf, T_w): every far-field condition whose state equals
 * that of the first far-field condition becomes the Maxwellian of density
 * rho_inf moving at speed U_inf along that state's velocity direction (x if it
 * is at rest) at that state's temperature; every diffuse wall whose tag is in
 * wall_tags gets temperature T_w.  theta == NULL evaluates at the simulation's
 * own values.  out[0] = J at theta, out[1..3] = dJ/dtheta by the hand-written
 * reverse sweep (face states recomputed from per-step checkpoints of W).
 * The recorded particle data never depend on theta.  At order 2 the
 * limiter values of each step are those of the frozen forward at theta and are
 * held fixed in the derivative (a frozen limiter); the far-field ghosts of the
 * reconstruction hold the far-field state at theta.  K = 0 internal degrees
 * of freedom only (E_UNSUPPORTED otherwise); the scratch memory is the
 * caller's device workspace of at least ugkwp_adjoint_query bytes (256-byte
 * aligned). */
typedef struct {
    int32_t functional;          /* 0 drag, 1 wall heat flux */
    int32_t n_steps;             /* K >= 1 */
    const int32_t* wall_tags;    /* host array of boundary tags */
    int32_t n_wall_tags;
    int32_t reserved_;
    const double* theta;         /* host [3] or NULL */
    void* d_workspace;
    size_t workspace_bytes;
} ugkwp_adjoint_req;
int ugkwp_adjoint_query(const ugkwp_sim* s, int32_t n_steps, size_t* bytes);
int ugkwp_adjoint_wave(ugkwp_sim* s, const ugkwp_adjoint_req* r, double* out);

/* Time step without any device allocation (this library's addition; the
 * paper has no counterpart).  Some callers cannot call cudaMalloc or hand the
 * library a workspace: a solver embedded in a host application that reserves
 * all device memory for itself up front, a plug-in whose framework forbids
 * allocation, or a latency-critical loop that must never wait on an allocator.
 * For them this entry point computes the time step of one UGKWP step,
 *   dt = CFL min_i |Omega_i| / sum_d (|U_d| + 3 sqrt(R T_i)) DeltaS_i^d
 * (Sec. 2.4 (a)), from device arrays the caller already owns, and writes it
 * to d_dt[0] on the given stream (cudaStream_t, NULL = legacy default stream).
 *   d_W   [5][n_cells] conservative variables (rho, rho U, rho E) of a
 *         monatomic gas (K = 0: p = (rho E - rho |U|^2/2) / 1.5), device
 *   d_vol [n_cells] cell volumes, device
 *   d_dS  [3][n_cells] projected areas DeltaS^x, ^y, ^z, device
 * Cells with rho <= 0 or p <= 0 are skipped; if no cell is valid d_dt[0] is
 * +inf.  The partial minima live in one array of static device memory of
 * UGKWP_NOALLOC_MAX_CELLS / 256 doubles (512 KiB) that every GPU which loads
 * the library holds until the process exits; n_cells above
 * UGKWP_NOALLOC_MAX_CELLS is rejected with UGKWP_E_ARG.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The address
 * is kept for the life of the process: after cudaDeviceReset (or anything else
 * that destroys the device's primary context) it is stale, so do not call this
 * entry point on that device again in the same process.  Every call
 * shares the array and leaves its contents behind (each call writes every slot
 * it reads, so nothing needs clearing): calls whose work overlaps on the GPU,
 * on any streams, race and must be ordered by the caller.  The call returns
 * once its two kernels are enqueued; it allocates no memory and does not
 * synchronise.  Errors: UGKWP_E_ARG, UGKWP_E_CUDA. */
#define UGKWP_NOALLOC_MAX_CELLS (1 << 24)
int ugkwp_time_step_noalloc(const double* d_W, const double* d_vol, const double* d_dS, int32_t n_cells,
                            double R, double CFL, double* d_dt, void* cuda_stream);

/* Copy the calling thread's last error message (NUL-terminated) into buf. */
int ugkwp_last_error(char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* UGKWP_H */
