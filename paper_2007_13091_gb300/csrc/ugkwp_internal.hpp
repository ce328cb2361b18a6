// Internal types of the ugkwp library: host mesh object, device views passed
// to the kernels by value, and the launch functions of each kernel family.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ugkwp.h"

namespace ugkwp {

// Error bits of the device error word.
enum : int32_t {
    ERRB_CAPACITY = 1,
    ERRB_TRACK_LIMIT = 2,
    ERRB_FIXED_OVERFLOW = 4,
    ERRB_NONFINITE = 8,
    ERRB_SAMPLE_LIMIT = 16,
    ERRB_SORT = 64,         // a cell holds more survivors than its count (sort skipped them)
    ERRB_CHECK = 128,       // a kernel's own bounds or alignment check failed (the access was skipped;
                            // CNT_CHECK holds the check and the value)
};

// Largest tile of the tracking kernel (particles per block and tile); the
// particle arrays hold whole tiles of this size.
constexpr int TRACK_TILE_MAX = 256;

// Device counters (int64 slots).  The counters that tracking blocks update
// with atomics sit on 128-byte lines of their own.
enum : int {
    CNT_N_A = 0,        // slots of the current buffer before the samples: the last step's
                        // survivor buckets (holes marked by cell -1) and overflow slots
    CNT_N_B = 1,        // slots tracked this step (N_A + samples), from the scan
    CNT_SURV = 2,       // survivors of the last step (particles alive)
    CNT_SAMPLED = 3,
    CNT_COLLIDED = 4,
    CNT_EXITED = 5,
    CNT_LOST = 6,
    CNT_CROSSINGS = 7,
    CNT_WALL = 8,
    CNT_STEP = 9,       // step index of the next step
    CNT_TRACKED = 10,
    CNT_DT_BITS = 11,   // min_i |Omega_i| / sum Lambda as ordered bits (positive double)
    CNT_ERR = 12,       // error bits
    CNT_MOVES = 13,     // particle moves since init (never reset by a step)
    CNT_NSAM = 14,      // particles sampled this step (from the scan)
    CNT_WTOT = 15,      // slots of the survivor buckets of the buffer written this step (from the scan)
    CNT_RESV = 16,      // mover slots reserved this step
    CNT_TILE = 32,      // next grab of tracking tiles
    CNT_IMPORT = 40,    // a state import's first failed particle: (index << 3) | problem
    CNT_OVF = 48,       // overflow slots (survivors whose bucket is full) taken this step
    CNT_CHECK = 56,     // the first failed self-check: (check << 48) | value
    CNT_SLOTS = 64,
};
// Tiles taken from the tile counter per atomic.
constexpr int TILE_GRAB = 4;

struct DevBc {
    int32_t type;
    int32_t pad;
    double T_w;
    double U_w[3];
    double W_in[5];
    float c2rt_f;  // binary32 rounding of -2 R T_w (mixed-mode wall emission)
    float sw_f;    // binary32 rounding of sqrt(R T_w)
};

struct DevParams {
    double R, mu_ref, T_ref, omega, CFL, C2;
    double pr_fix;         // 1/Pr - 1: factor of the equilibrium heat flux added to the energy flux (0: BGK)
    int32_t N_ref, N_min, max_crossings, precision;
    int32_t order;
    int32_t sampling;      // UGKWP_SAMPLE_*
    int32_t averaging;     // add dt W^{n+1} to the time-average sums
    int32_t gks;           // 0: UGKWP step; 1: GKS step (no particles); 2: GKS step, local time steps
    int32_t K;             // internal degrees of freedom
    int32_t kpad_;
    uint64_t seed;
    int64_t capacity;
    int32_t exps[5];
    int32_t n_bc;
    double qscale[5];      // 2^e (fixed-point quantum)
    double qinv[5];        // 2^-e
    DevBc bc[16];
};

// Tracking record of one tet: outward face planes (n, d) and neighbour codes
// (tet << 2 | local face in the neighbour, or -1 - boundary-face index).  The
// binary32 record (mixed mode, positions relative to the tet's anchor) adds,
// per local face k, the anchor of this tet minus the anchor of the neighbour
// across k at da[3k..3k+2] (exact in binary32; 0 at boundary faces): one
// 128-byte line per tet.
struct __align__(128) TrkF {
    float4 pl[4];
    int4 nb;
    float da[12];
};
struct __align__(16) Dbl4 {
    double x, y, z, w;
};
struct __align__(16) TrkD {
    Dbl4 pl[4];
    int4 nb;
};

struct DevMesh {
    int32_t nc, nf, nbf;
    int32_t nif;             // interior faces (they lead face_order)
    const double* vol;       // [nc]
    const double* ivol;      // [nc] 1 / vol
    const double* dS;        // [3][nc]
    const double* vtx;       // [12][nc]: vertex k coordinate c at [(3k+c) nc + i]
    const int32_t* cf;       // [4][nc] face of local face k
    const int32_t* cfs;      // [nc] bit k set if the cell owns local face k
    const TrkF* trk_f;       // [nc]
    const TrkD* trk_d;       // [nc]
    const float* smp_f;      // [24][nc] mixed mode: for coordinate c at [(8c + j) nc + i], j = 0, 1: vertex 0
                             // minus the tet's anchor, j = 2k, 2k + 1 (k = 1..3): edge p_k - p_0, each
                             // binary64 value split into a binary32 pair (high, low)
    const float* bf_f;       // [11][nbf] mixed mode: n, t1, t2, U_w.t1, U_w.t2 of each boundary face, binary32
    // second-order reconstruction (order 2)
    const double* lsq_c;     // [12][nc]: gradient = sum_k c_k (v_k - v_i), c_k at [(3k+d) nc + i]
    const double* lsq_dxf;   // [12][nc]: face centroid minus cell centroid for local face k
    const double* eps2;      // [nc] Venkatakrishnan epsilon^2 = (K h)^3
    const int32_t* f_lk;     // [nf] owner's local face | neighbour's local face << 2
    const int32_t* face_order;  // [nf] interior faces, then boundary faces grouped by type
    const int32_t* f_own;    // [nf]
    const int32_t* f_nbr;    // [nf] >= 0 tet, else -1 - boundary index
    const double* f_n;       // [3][nf]
    const double* f_area;    // [nf]
    const int32_t* bf_tag;   // [nbf]
    const double* bf_n;      // [3][nbf] outward unit normal (double)
    const double* bf_t1;     // [3][nbf]
    const double* bf_t2;     // [3][nbf]
};

template <class Real> struct PartView {
    Real* x[3];
    Real* u[3];
    double* m;
    int32_t* cell;
    uint64_t* id;
    Real* e;   // internal energy (K > 0; NULL otherwise)
    Real* e2;  // mover list only: internal energy at the end
};

struct PartBufRaw {
    void* x[3];
    void* u[3];
    double* m;
    int32_t* cell;
    uint64_t* id;
    void* e;
    void* e2;
};

struct DevState {
    double* W;            // [5][nc]
    double* prim;         // [5][nc] rho, Ux, Uy, Uz, T
    double* tau;          // [nc]
    float* tauf;          // [nc] binary32 rounding of tau (MIXED t_f draw)
    float4* usig;         // [nc] binary32 roundings of U and the sampling spread (MIXED sampling)
    double* sig;          // [nc] sampling spread s sqrt(RT) of energy-matched sampling
    double* dtc;          // [nc] local time step CFL |Omega| / sum_d Lambda^d (GKS step, local steps)
    double* gpc;          // [GP_NC][nc] first-order g_p: acceptance polynomial and bound per cell
    double* wsum;         // [5][nc] time-average sums of dt^n W^n
    double* tsum;         // [1] sum of dt^n
    double* rhoh;         // [nc]
    double* rhop;         // [nc]
    int32_t* nsam;        // [nc]
    double* msam;         // [nc]
    int32_t* nleft;       // [nc] survivors at the start of the step
    int32_t* nleft_next;  // [nc]
    int64_t* smass;       // [nc] survivors' fixed-point mass
    int64_t* smass_next;  // [nc]
    int32_t* cnt;         // [nc] particles per cell after sampling
    int32_t* soff;        // [nc] exclusive scan of N_sam (sampled-particle index)
    int32_t* wcap;        // [nc] slots of the cell's survivor bucket in the buffer written this step
    int32_t* woff;        // [nc] first slot of that bucket (exclusive scan of wcap); the bucket's
                          // fill count is nleft_next (the survivors that ended in the cell)
    int64_t* pflux;       // [5][nc] fixed-point particle flux
    int64_t* wacc;        // [5][nc] fixed-point scratch for W^p
    double* mom;          // [5][nc] staging of moments copied to the host
    double* F;            // [5][nf]
    double* gradW;        // [15][nc] limited gradients of W, [(3q+d) nc + i] (order 2)
    double* gradH;        // [3][nc] limited gradient of rho^h (order 2)
    int2* bsum;           // [n_scan_blocks] block sums of (count, N_sam)
    double* t;            // [1]
    double* dt;           // [1]
    int64_t* cnt64;       // [CNT_SLOTS]
};

// One member of a fused batch: a simulation's device structures for one step,
// with its particle buffers in this step's roles.
struct BatchMember {
    DevMesh m;
    DevState s;
    DevParams p;
    PartBufRaw a;   // this step's particles
    PartBufRaw b;   // the buffer the survivors are written to
    PartBufRaw mv;  // the movers
};

// The block a kernel body runs as: its index among the blocks that work on
// the same simulation, and their number (blockIdx.x and gridDim.x of a launch
// for one simulation).
struct Blk {
    int id, n;
};

struct MeshHost {
    int32_t nn = 0, nc = 0, nf = 0, nbf = 0;
    std::vector<double> xyz;
    std::vector<int32_t> tet;
    std::vector<int32_t> cf;       // [4*nc] face of local face k (cell-major)
    std::vector<int8_t> cf_sign;   // [4*nc]
    std::vector<int32_t> f_own, f_own_k, f_nbr, f_nbr_k, f_tag;  // f_nbr < 0 for boundary
    std::vector<double> f_n, f_area, f_d, f_t1, f_t2, f_c;       // [3*nf] / [nf]
    std::vector<double> vol, dS;                                 // [nc], [3*nc]
    std::vector<int32_t> bf_of_face;                             // [nf] boundary index or -1
    std::vector<int32_t> face_of_bf;                             // [nbf]
};

// First-order g_p sampling: per cell phi(X) = a0 + L.X + X^T Q X + (C.X)|X|^2
// of X = (u - U)/sqrt(RT) and the acceptance bound M:
// [a0, L(3), Qxx, Qyy, Qzz, Qxy, Qxz, Qyz, C(3), M].
constexpr int GP_NC = 14;
constexpr int GP_ATTEMPTS = 64;

// Kernel launchers (stream-ordered, no synchronisation).
// cells per block of the counting and offset kernels (256: every SM takes
// blocks on a ~1e5-cell mesh), and threads of the one-block scan of their
// block sums
constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_SUM_THREADS = 1024;
__host__ __device__ inline int scan_blocks(int nc) { return (nc + SCAN_BLOCK - 1) / SCAN_BLOCK; }

void launch_reset(const DevMesh& m, const DevState& s, cudaStream_t st);
void launch_cell_prep(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st);
void launch_sample_count(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st);
void launch_scan(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st);
// Grid sizes of the step kernels that loop over their work (any positive
// value gives the same results; chosen for speed, e.g. by the autotuner).
// Shape of the tracking kernel: threads (= particles) per block and tile.
struct TrackShape {
    int threads;  // 128 or 256
};
struct LaunchCfg {
    int particle_blocks;  // blocks of the sampling, tracking and movers kernels
    int wave_blocks;      // blocks of the persistent second-order wave kernels
    TrackShape track;     // tracking kernel shape
    int carveout;         // preferred shared-memory carveout (percent) of the step's kernels, -1: driver default
};

void launch_sample_write(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& b,
                         int blocks, cudaStream_t st);
// Energy-matched sampling: the per-cell spread s sqrt(RT) (sig, usig.w).
void launch_sample_scale(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st);
// Tracking of buffer b (survivors, then this step's samples); the survivors go
// compacted to nxt, the particles whose counting flux is non-zero are listed in
// movers and their flux added by launch_movers.
void launch_track(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& b,
                  const PartBufRaw& nxt, const PartBufRaw& movers, const TrackShape& sh, int blocks, cudaStream_t st);
// The common preferred shared-memory carveout of the step's kernels (a
// kernel attribute): set outside stream capture, before the configuration's
// first launch.
cudaError_t configure_particle_kernels(const DevParams& p, int carveout);
cudaError_t configure_wave_kernels(int carveout);
cudaError_t configure_cell_kernels(int carveout);
void launch_movers(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& a,
                   int blocks, cudaStream_t st);

// First-order flux of face_order[first..nf); second-order flux of the nif interior faces.
void launch_face_flux(const DevMesh& m, const DevState& s, const DevParams& p, int first, int blocks,
                      cudaStream_t st);
void launch_face_flux_o2(const DevMesh& m, const DevState& s, const DevParams& p, int blocks, cudaStream_t st);
void launch_gradients(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st);
void launch_gp_coef(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st);
// a10, and the end of a11: the unused slots of each survivor bucket of the
// buffer written this step (cell array wcell) are marked as holes.
void launch_cell_update(const DevMesh& m, const DevState& s, const DevParams& p, int32_t* wcell, cudaStream_t st);
// the wave part of a step's update (before the particle part of launch_cell_update)
void launch_wave_update(const DevMesh& m, const DevState& s, cudaStream_t st);
// Survivor bucket of a cell that starts a step with `cnt` particles: the slots
// the next buffer reserves for the survivors that end the step in it.
__host__ __device__ inline int bucket_slots(int cnt) { return cnt + cnt / 32 + 4; }
void launch_rebuild_survivors(const DevMesh& m, const DevState& s, const DevParams& p,
                              const PartBufRaw& a, cudaStream_t st);
// checks a state image's particles in the spare buffer b and, with convert
// (mixed mode, binary64 image), converts x, u, e from the binary64 staging
// xs, us, es into it (anchors anc [nc][3])
void launch_import(int nc, long long n, bool mixed, bool convert, const double* anc, const double* xs,
                   const double* us, const double* es, const PartBufRaw& b, unsigned long long* err,
                   cudaStream_t st);
void launch_wp_moments(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& a,
                       double* out, cudaStream_t st);
void launch_prim_moments(const DevMesh& m, const DevState& s, const DevParams& p, int which,
                         double* out, cudaStream_t st);
void launch_wbar(const DevMesh& m, const DevState& s, double* out, cudaStream_t st);
void launch_kn_gll(const DevMesh& m, const DevState& s, const DevParams& p, double* out, cudaStream_t st);

// ---- fused batches: one launch of each step kernel for a chunk of up to
// BATCH_CHUNK members of a batch that share precision, order, K and sampling.
// The chunk travels as the launch's parameter (read-only, like a single
// simulation's structures).  Kernels over cells or faces give member i the
// blocks off[cls][i] .. off[cls][i + 1] - 1 of the grid, on which it runs the
// body its own launch would run; the particle kernels (sampling, tracking,
// movers) take every member in turn on the whole grid.
constexpr int BATCH_CHUNK = 13;
enum BatchClass { BCL_RESET, BCL_CELLS, BCL_SCAN, BCL_GRAD, BCL_GPC, BCL_FLUX_O2, BCL_FLUX, BCL_N };
struct BatchChunk {
    int32_t n;
    int32_t off[BCL_N][BATCH_CHUNK + 1];
    BatchMember mem[BATCH_CHUNK];
};
static_assert(sizeof(BatchChunk) <= 32764, "a chunk must fit a launch's parameter space");
int blocks_reset(int nc);        // grid of one simulation's reset launch
int blocks_cells(int nc);        // one thread per cell, 256 per block
int blocks_gp_coef(int nc);      // one thread per cell, 128 per block
int gradient_threads();          // threads per block of the gradient kernel
void launch_reset_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_cell_prep_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_sample_count_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_scan_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_cell_update_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_wave_update_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_gradients_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_gp_coef_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_face_flux_o2_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_face_flux_batch(const BatchChunk& c, int blocks, cudaStream_t st);
void launch_sample_scale_batch(const BatchChunk& c, int blocks, int precision, cudaStream_t st);
void launch_sample_write_batch(const BatchChunk& c, int blocks, int precision, cudaStream_t st);
void launch_track_batch(const BatchChunk& c, int precision, bool ke, const TrackShape& sh, int blocks,
                        cudaStream_t st);
void launch_movers_batch(const BatchChunk& c, int blocks, int precision, cudaStream_t st);

// ---- adjoint of the frozen-particle wave map (first order)
struct AdjBc {
    int32_t param_ff;    // far-field state replaced by theta (rho_inf, U_inf)
    int32_t param_wall;  // diffuse-wall temperature replaced by theta[2]
    int32_t listed;      // boundary faces with this tag enter the functional
    int32_t pad;
    double e[3];         // direction of the parameterised far-field velocity
    double RT;           // its R T (kept)
};
struct AdjParams {
    AdjBc b[16];
    int32_t comp;        // 1: x momentum (drag), 4: energy (wall heat flux)
    int32_t pad;
};
void launch_adj_record(const DevMesh& m, const DevState& s, const DevParams& p, double* rho_p, double* pf,
                       cudaStream_t st);
// Second order: the step's limiter values phi [6][nc] (recorded by the forward
// pass, used by the reverse one) and scratch: limited gradients gW [15][nc],
// gH [3][nc], the faces' products with both cells' gradients gbar [36][nf],
// phi times their per-cell sums gg [18][nc], far-field ghost products thc [3][nc].
struct AdjO2 {
    double* phi;
    double* gW;
    double* gH;
    double* gbar;
    double* gg;
    double* thc;
};
// Fluxes at theta, the step's functional term Jn[0] and the next state Wn.
void launch_adj_forward(const DevMesh& m, const DevParams& p, const AdjParams& ap, const double* W, const double* rho_p,
                        const double* pf, double dt, const double* theta, const AdjO2& o2, double* F, double* jf,
                        double* Jn, double* Wn, cudaStream_t st);
// lambda^n from lambda^{n+1} and this step's dJ/dtheta terms th_out[3].
void launch_adj_reverse(const DevMesh& m, const DevParams& p, const AdjParams& ap, const double* W,
                        const double* rho_p, double dt, const double* theta, const AdjO2& o2, const double* lam_next,
                        double* lam, double* wbar, double* thbar, double* th_out, cudaStream_t st);

int sm_count();       // multiprocessors of the current device
int particle_grid();  // default grid of particle kernels (8 blocks per SM)
int wave_threads();   // threads per block of the persistent wave kernels

}  // namespace ugkwp
