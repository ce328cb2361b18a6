// C-ABI of the ugkwp library (declared in include/ugkwp.h): argument checks,
// workspace layout, host-side preparation of the device geometry, the order of
// kernel launches of one step, and state import/export.
// This file is compiled with floating-point contraction disabled.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "ugkwp_internal.hpp"

namespace ugkwp {
bool build_mesh(const ugkwp_mesh_desc& d, MeshHost& M, std::string& err);
}

using namespace ugkwp;

struct ugkwp_mesh {
    MeshHost h;
};

struct TimedLaunch {
    int k;
    cudaEvent_t a, b;
};

struct ugkwp_sim {
    DevParams P;
    DevMesh M;
    DevState S;
    PartBufRaw A, B;   // A: the current particles (between steps: the survivors); B: the next survivors
    PartBufRaw Mv;     // the step's movers (particles whose counting flux is non-zero)
    std::vector<double> anchor;  // [3*nc] anchors of the tets (mixed mode; 0 in binary64)
    cudaStream_t stream = nullptr;
    // device staging of ugkwp_import_state in mixed mode (the tets' anchors
    // and the image's binary64 positions, velocities and internal energies),
    // kept between imports
    void* imp = nullptr;
    size_t imp_bytes = 0;
    int64_t step = 0;
    int32_t n_bc = 0;
    size_t real_size = 8;
    int64_t capacity = 0;
    bool timing = false;
    int64_t launches[UGKWP_N_KERNELS] = {};
    std::vector<TimedLaunch> pending;
    std::vector<cudaEvent_t> pool;
    // the wave flux (binary64-bound) runs beside the particle kernels; the
    // second half of the tracking grid joins from `aux` once the wave is done
    cudaStream_t wave = nullptr, aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, sampled = nullptr, tracked = nullptr, gp_ready = nullptr,
                waved = nullptr;
    // grid sizes of the looping step kernels
    LaunchCfg lc{0, 0, {128}, -1};
    // two-step CUDA graphs, one per ping-pong parity (keyed by buffer A), with
    // the kernels each one launches per class
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    void* graph_key[2] = {nullptr, nullptr};
    int64_t graph_launches[2][UGKWP_N_KERNELS] = {};
    bool graphs_ok = true;
    // counts the changes of the structures the kernels receive by value
    // (parameters, launch configuration, buffers): a batch's graphs check it
    uint64_t gen = 0;
    void drop_graphs() {
        ++gen;
        for (int k = 0; k < 2; ++k) {
            if (graph[k]) cudaGraphExecDestroy(graph[k]);
            graph[k] = nullptr;
            graph_key[k] = nullptr;
        }
    }
    ~ugkwp_sim() {
        drop_graphs();
        for (auto& t : pending) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
        for (auto e : pool) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (sampled) cudaEventDestroy(sampled);
        if (tracked) cudaEventDestroy(tracked);
        if (gp_ready) cudaEventDestroy(gp_ready);
        if (waved) cudaEventDestroy(waved);
        if (imp) cudaFree(imp);
        if (wave) cudaStreamDestroy(wave);
        if (aux) cudaStreamDestroy(aux);
    }
};

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

}  // namespace

namespace ugkwp {
void set_last_error_message(const std::string& msg) { g_err = msg; }
}

namespace {

int cuda_fail(cudaError_t e, const char* where) {
    return fail(UGKWP_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CU(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

// Linear allocator over the caller's workspace (256-byte aligned chunks).
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base((char*)b) {}
    template <class T> T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

void layout(const MeshHost& mh, int64_t cap, size_t rs, bool with_e, Carver& c, DevMesh& M, DevState& S,
            PartBufRaw& A, PartBufRaw& B, PartBufRaw& Mv) {
    const size_t nc = mh.nc, nf = mh.nf, nbf = mh.nbf;
    M.nc = mh.nc; M.nf = mh.nf; M.nbf = mh.nbf; M.nif = mh.nf - mh.nbf;
    M.vol = c.take<double>(nc);
    M.ivol = c.take<double>(nc);
    M.dS = c.take<double>(3 * nc);
    M.vtx = c.take<double>(12 * nc);
    M.cf = c.take<int32_t>(4 * nc);
    M.cfs = c.take<int32_t>(nc);
    M.trk_f = nullptr;
    M.trk_d = nullptr;
    if (rs == 4) M.trk_f = c.take<TrkF>(nc);
    else M.trk_d = c.take<TrkD>(nc);
    M.face_order = c.take<int32_t>(nf);
    M.smp_f = c.take<float>(24 * nc);
    M.bf_f = c.take<float>(11 * (nbf ? nbf : 1));
    M.lsq_c = c.take<double>(12 * nc);
    M.lsq_dxf = c.take<double>(12 * nc);
    M.eps2 = c.take<double>(nc);
    M.f_lk = c.take<int32_t>(nf);
    M.f_own = c.take<int32_t>(nf);
    M.f_nbr = c.take<int32_t>(nf);
    M.f_n = c.take<double>(3 * nf);
    M.f_area = c.take<double>(nf);
    M.bf_tag = c.take<int32_t>(nbf ? nbf : 1);
    M.bf_n = c.take<double>(3 * (nbf ? nbf : 1));
    M.bf_t1 = c.take<double>(3 * (nbf ? nbf : 1));
    M.bf_t2 = c.take<double>(3 * (nbf ? nbf : 1));
    S.W = c.take<double>(5 * nc);
    S.prim = c.take<double>(5 * nc);
    S.tau = c.take<double>(nc);
    S.tauf = c.take<float>(nc);
    S.usig = c.take<float4>(nc);
    S.sig = c.take<double>(nc);
    S.dtc = c.take<double>(nc);
    S.gpc = c.take<double>((size_t)GP_NC * nc);
    S.wsum = c.take<double>(5 * nc);
    S.tsum = c.take<double>(1);
    S.rhoh = c.take<double>(nc);
    S.rhop = c.take<double>(nc);
    S.nsam = c.take<int32_t>(nc);
    S.msam = c.take<double>(nc);
    S.nleft = c.take<int32_t>(nc);
    S.nleft_next = c.take<int32_t>(nc);
    S.smass = c.take<int64_t>(nc);
    S.smass_next = c.take<int64_t>(nc);
    S.cnt = c.take<int32_t>(nc);
    S.soff = c.take<int32_t>(nc);
    S.wcap = c.take<int32_t>(nc);
    S.woff = c.take<int32_t>(nc);
    S.pflux = c.take<int64_t>(5 * nc);
    S.wacc = c.take<int64_t>(5 * nc);
    S.mom = c.take<double>(5 * nc);
    S.F = c.take<double>(5 * nf);
    S.gradW = c.take<double>(15 * nc);
    S.gradH = c.take<double>(3 * nc);
    S.bsum = c.take<int2>((size_t)scan_blocks(mh.nc) + 1);
    S.t = c.take<double>(1);
    S.dt = c.take<double>(1);
    S.cnt64 = c.take<int64_t>(CNT_SLOTS);
    // each particle array holds the capacity rounded up to whole tiles of the
    // tracking kernel (TRACK_TILE_MAX particles), so that a tile's loads of
    // its whole slots stay inside the array
    const size_t capt = ((size_t)cap + TRACK_TILE_MAX - 1) / TRACK_TILE_MAX * TRACK_TILE_MAX;
    for (PartBufRaw* pb : {&A, &B, &Mv}) {
        for (int d = 0; d < 3; ++d) pb->x[d] = c.take<char>(rs * capt);
        for (int d = 0; d < 3; ++d) pb->u[d] = c.take<char>(rs * capt);
        pb->m = c.take<double>(capt);
        pb->cell = c.take<int32_t>(capt);
        pb->id = c.take<uint64_t>(capt);
        pb->e = with_e ? (void*)c.take<char>(rs * capt) : nullptr;
        pb->e2 = (with_e && pb == &Mv) ? (void*)c.take<char>(rs * capt) : nullptr;
    }
}

int check_params(const ugkwp_params* p, const MeshHost* mh) {
    if (!p) return fail(UGKWP_E_ARG, "params is NULL");
    if (!(p->R > 0.0) || !(p->mu_ref > 0.0) || !(p->T_ref > 0.0) || !std::isfinite(p->omega))
        return fail(UGKWP_E_ARG, "R, mu_ref and T_ref must be positive and omega finite");
    if (!(p->CFL > 0.0 && p->CFL <= 1.0)) return fail(UGKWP_E_ARG, "CFL must be in (0, 1]");
    if (!(p->C2 >= 0.0)) return fail(UGKWP_E_ARG, "C2 must be >= 0");
    if (!(p->Pr >= 0.0) || !std::isfinite(p->Pr)) return fail(UGKWP_E_ARG, "Pr must be finite and >= 0 (0: BGK)");
    if (p->order != 1 && p->order != 2) return fail(UGKWP_E_ARG, "order must be 1 or 2");
    if (p->order == 2 && !(p->venkat_K >= 0.0)) return fail(UGKWP_E_ARG, "venkat_K must be >= 0");
    if (p->N_ref <= 0 || p->N_min < 0) return fail(UGKWP_E_ARG, "N_ref must be > 0 and N_min >= 0");
    if (p->precision != UGKWP_FP64 && p->precision != UGKWP_MIXED) return fail(UGKWP_E_ARG, "unknown precision");
    if (p->max_crossings <= 0) return fail(UGKWP_E_ARG, "max_crossings must be > 0");
    if (p->sampling != UGKWP_SAMPLE_MAXWELL && p->sampling != UGKWP_SAMPLE_ENERGY_MATCHED &&
        p->sampling != UGKWP_SAMPLE_GP1)
        return fail(UGKWP_E_ARG, "unknown sampling mode");
    if (p->K < 0 || p->K > 8) return fail(UGKWP_E_ARG, "K must be in [0, 8]");
    if (p->K > 0 && p->sampling != UGKWP_SAMPLE_MAXWELL)
        return fail(UGKWP_E_ARG, "internal degrees of freedom (K > 0) need UGKWP_SAMPLE_MAXWELL");
    if (p->sampling == UGKWP_SAMPLE_GP1 && p->order != 2)
        return fail(UGKWP_E_ARG, "first-order g_p sampling needs order 2 (the cell slopes)");
    if (p->particle_capacity < 0 || p->particle_capacity >= ((int64_t)1 << 31))
        return fail(UGKWP_E_ARG, "particle_capacity must be in [0, 2^31)");
    if (p->n_bc < 0 || p->n_bc > 16) return fail(UGKWP_E_ARG, "n_bc must be in [0, 16]");
    for (int b = 0; b < p->n_bc; ++b) {
        const ugkwp_bc& bc = p->bc[b];
        if (bc.type < 1 || bc.type > 4) return fail(UGKWP_E_ARG, "unknown boundary type in bc[" + std::to_string(b) + "]");
        if (bc.type == UGKWP_BC_DIFFUSE_WALL && !(bc.T_w > 0.0)) return fail(UGKWP_E_ARG, "wall temperature must be > 0");
        if (bc.type == UGKWP_BC_FARFIELD) {
            const double* W = bc.W_in;
            const double rho = W[0];
            if (!(rho > 0.0)) return fail(UGKWP_E_ARG, "far-field density must be > 0");
            const double U2 = ((W[1] / rho) * (W[1] / rho) + (W[2] / rho) * (W[2] / rho)) + (W[3] / rho) * (W[3] / rho);
            if (!((W[4] - 0.5 * (rho * U2)) > 0.0)) return fail(UGKWP_E_ARG, "far-field pressure must be > 0");
        }
    }
    if (mh) {
        for (int f = 0; f < mh->nf; ++f)
            if (mh->f_nbr[f] < 0 && mh->f_tag[f] >= p->n_bc)
                return fail(UGKWP_E_ARG, "boundary tag " + std::to_string(mh->f_tag[f]) + " has no entry in params.bc");
    }
    return UGKWP_OK;
}

int ceil_log2(double b) {
    int ex;
    const double mant = std::frexp(b, &ex);
    return mant == 0.5 ? ex - 1 : ex;
}

// Fixed-point quanta 2^e_q: e_q = ceil(log2 B_q) - 50 with B_mass the largest
// cell mass, B_mom = B_mass c, B_E = B_mass c^2 / 2, c the largest |U| + 5 sqrt(RT)
// over the cells and the wall / far-field states, with p = (rho E - rho |U|^2 / 2)
// / ((3 + K) / 2) for K internal degrees of freedom.
void fixed_point_exponents(const MeshHost& mh, const ugkwp_params& p, const double* W, int32_t e[5]) {
    const int nc = mh.nc;
    double bm = 0.0, cmax = 0.0;
    auto speed = [&](const double* Wv, size_t stride) {
        const double rho = Wv[0];
        const double U[3] = {Wv[stride] / rho, Wv[2 * stride] / rho, Wv[3 * stride] / rho};
        const double U2 = (U[0] * U[0] + U[1] * U[1]) + U[2] * U[2];
        const double pr = (Wv[4 * stride] - 0.5 * (rho * U2)) / (1.5 + 0.5 * (double)p.K);
        const double T = pr / (rho * p.R);
        return std::sqrt((U[0] * U[0] + U[1] * U[1]) + U[2] * U[2]) + 5.0 * std::sqrt(p.R * T);
    };
    for (int i = 0; i < nc; ++i) {
        const double mass = W[i] * mh.vol[i];
        if (mass > bm) bm = mass;
        const double c = speed(W + i, (size_t)nc);
        if (c > cmax) cmax = c;
    }
    for (int b = 0; b < p.n_bc; ++b) {
        const ugkwp_bc& bc = p.bc[b];
        double c = 0.0;
        if (bc.type == UGKWP_BC_DIFFUSE_WALL)
            c = std::sqrt((bc.U_w[0] * bc.U_w[0] + bc.U_w[1] * bc.U_w[1]) + bc.U_w[2] * bc.U_w[2]) + 5.0 * std::sqrt(p.R * bc.T_w);
        else if (bc.type == UGKWP_BC_FARFIELD)
            c = speed(bc.W_in, 1);
        if (c > cmax) cmax = c;
    }
    e[0] = ceil_log2(bm) - 50;
    e[1] = e[2] = e[3] = ceil_log2(bm * cmax) - 50;
    e[4] = ceil_log2(bm * cmax * cmax * 0.5) - 50;
}

void set_exps(DevParams& P, const int32_t e[5]) {
    for (int q = 0; q < 5; ++q) {
        P.exps[q] = e[q];
        P.qscale[q] = std::ldexp(1.0, e[q]);
        P.qinv[q] = std::ldexp(1.0, -e[q]);
    }
}

// Kernel attributes of a launch configuration (set outside stream capture).
cudaError_t configure_kernels(const DevParams& P, const LaunchCfg& lc) {
    cudaError_t e = configure_particle_kernels(P, lc.carveout);
    if (e == cudaSuccess) e = configure_wave_kernels(lc.carveout);
    if (e == cudaSuccess) e = configure_cell_kernels(lc.carveout);
    return e;
}

int read_error(ugkwp_sim* s) {
    int64_t h[CNT_SLOTS];
    CU(cudaMemcpyAsync(h, s->S.cnt64, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    const int64_t e = h[CNT_ERR];
    if (!e) return UGKWP_OK;
    const int64_t zero = 0;
    CU(cudaMemcpyAsync(s->S.cnt64 + CNT_ERR, &zero, sizeof(zero), cudaMemcpyHostToDevice, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    if (e & ERRB_CAPACITY) return fail(UGKWP_E_CAPACITY, "particle capacity exceeded: the step's particle writes were skipped and the particle state is no longer valid");
    if (e & ERRB_NONFINITE) return fail(UGKWP_E_NONFINITE, "non-positive density or pressure in a cell");
    if (e & ERRB_TRACK_LIMIT) return fail(UGKWP_E_TRACK_LIMIT, std::to_string(h[CNT_LOST]) + " particles exceeded max_crossings");
    if (e & ERRB_FIXED_OVERFLOW) return fail(UGKWP_E_FIXED_OVERFLOW, "fixed-point particle flux overflow");
    if (e & ERRB_SAMPLE_LIMIT) return fail(UGKWP_E_CAPACITY, "more than 65534 particles sampled in one cell");
    if (e & ERRB_SORT)
        return fail(UGKWP_E_STATE, "survivor counts per cell disagree with the survivors: the particle state is not valid");
    if (e & ERRB_CHECK)
        return fail(UGKWP_E_STATE, "a kernel's bounds or alignment check failed (check " + std::to_string(h[CNT_CHECK] >> 48) +
                                   ", value " + std::to_string(h[CNT_CHECK] & 0xffffffffffffLL) + "); the access was skipped");
    return fail(UGKWP_E_STATE, "device error word " + std::to_string(e));
}

}  // namespace

extern "C" {

int ugkwp_last_error(char* buf, size_t len) {
    if (!buf || len == 0) return UGKWP_E_ARG;
    std::snprintf(buf, len, "%s", g_err.c_str());
    return UGKWP_OK;
}

int ugkwp_mesh_load(const ugkwp_mesh_desc* d, ugkwp_mesh** out) {
    if (!d || !out) return fail(UGKWP_E_ARG, "NULL argument");
    *out = nullptr;
    if (d->n_nodes <= 0 || d->n_tets <= 0 || d->n_bfaces < 0 || !d->xyz || !d->tets ||
        (d->n_bfaces > 0 && (!d->bfaces || !d->bface_tags)))
        return fail(UGKWP_E_ARG, "invalid mesh description");
    if (d->n_tets >= (1 << 24)) return fail(UGKWP_E_ARG, "n_tets must be < 2^24");
    for (int32_t b = 0; b < d->n_bfaces; ++b)
        if (d->bface_tags[b] < 0 || d->bface_tags[b] >= 16) return fail(UGKWP_E_ARG, "boundary tags must be in [0, 16)");
    ugkwp_mesh* m = new ugkwp_mesh;
    std::string err;
    if (!build_mesh(*d, m->h, err)) {
        delete m;
        return fail(UGKWP_E_MESH, err);
    }
    *out = m;
    return UGKWP_OK;
}

int ugkwp_mesh_free(ugkwp_mesh* m) {
    delete m;
    return UGKWP_OK;
}

int ugkwp_query_sizes(const ugkwp_mesh* m, const ugkwp_params* p, ugkwp_sizes* out) {
    if (!m || !out) return fail(UGKWP_E_ARG, "NULL argument");
    int rc = check_params(p, &m->h);
    if (rc) return rc;
    DevMesh M{};
    DevState S{};
    PartBufRaw A{}, B{};
    Carver c(nullptr);
    PartBufRaw Mv{};
    layout(m->h, p->particle_capacity, p->precision == UGKWP_MIXED ? 4 : 8, p->K > 0, c, M, S, A, B, Mv);
    out->workspace_bytes = (c.off + 255) & ~(size_t)255;
    out->n_cells = m->h.nc;
    out->n_faces = m->h.nf;
    out->n_bfaces = m->h.nbf;
    return UGKWP_OK;
}

int ugkwp_init(const ugkwp_mesh* m, const ugkwp_params* p, const double* W0, void* d_workspace,
               size_t workspace_bytes, void* cuda_stream, ugkwp_sim** out) {
    if (!m || !W0 || !out) return fail(UGKWP_E_ARG, "NULL argument");
    *out = nullptr;
    int rc = check_params(p, &m->h);
    if (rc) return rc;
    const MeshHost& mh = m->h;
    const int nc = mh.nc, nf = mh.nf, nbf = mh.nbf;
    for (int i = 0; i < nc; ++i) {
        const double rho = W0[i];
        if (!(rho > 0.0) || !std::isfinite(rho)) return fail(UGKWP_E_NONFINITE, "W0 has rho <= 0 in cell " + std::to_string(i));
        const double U[3] = {W0[nc + i] / rho, W0[2 * nc + i] / rho, W0[3 * nc + i] / rho};
        const double pr = (W0[4 * nc + i] - 0.5 * (rho * ((U[0] * U[0] + U[1] * U[1]) + U[2] * U[2]))) / 1.5;
        if (!(pr > 0.0) || !std::isfinite(pr)) return fail(UGKWP_E_NONFINITE, "W0 has p <= 0 in cell " + std::to_string(i));
    }
    ugkwp_sizes sz;
    rc = ugkwp_query_sizes(m, p, &sz);
    if (rc) return rc;
    if (!d_workspace || workspace_bytes < sz.workspace_bytes)
        return fail(UGKWP_E_WORKSPACE, "workspace missing or smaller than ugkwp_query_sizes requires (" +
                                           std::to_string(sz.workspace_bytes) + " bytes)");
    if (((uintptr_t)d_workspace) & 255) return fail(UGKWP_E_WORKSPACE, "workspace must be 256-byte aligned");

    ugkwp_sim* s = new ugkwp_sim;
    s->stream = (cudaStream_t)cuda_stream;
    s->real_size = p->precision == UGKWP_MIXED ? 4 : 8;
    s->capacity = p->particle_capacity;
    s->n_bc = p->n_bc;
    Carver c(d_workspace);
    layout(mh, p->particle_capacity, s->real_size, p->K > 0, c, s->M, s->S, s->A, s->B, s->Mv);
    // parameters
    DevParams& P = s->P;
    std::memset(&P, 0, sizeof(P));
    P.R = p->R; P.mu_ref = p->mu_ref; P.T_ref = p->T_ref; P.omega = p->omega; P.CFL = p->CFL; P.C2 = p->C2;
    P.pr_fix = (p->Pr > 0.0 && p->Pr != 1.0) ? 1.0 / p->Pr - 1.0 : 0.0;
    P.N_ref = p->N_ref; P.N_min = p->N_min; P.max_crossings = p->max_crossings; P.precision = p->precision;
    P.order = p->order;
    P.sampling = p->sampling;
    P.K = p->K;
    P.seed = p->seed; P.capacity = p->particle_capacity; P.n_bc = p->n_bc;
    for (int b = 0; b < p->n_bc; ++b) {
        P.bc[b].type = p->bc[b].type;
        P.bc[b].T_w = p->bc[b].T_w;
        for (int k = 0; k < 3; ++k) P.bc[b].U_w[k] = p->bc[b].U_w[k];
        for (int k = 0; k < 5; ++k) P.bc[b].W_in[k] = p->bc[b].W_in[k];
        P.bc[b].c2rt_f = (float)(-2.0 * p->R * p->bc[b].T_w);
        P.bc[b].sw_f = (float)std::sqrt(p->R * p->bc[b].T_w);
    }
    int32_t e[5];
    fixed_point_exponents(mh, *p, W0, e);
    set_exps(P, e);
    // host images of the device geometry
    std::vector<double> dS(3 * (size_t)nc), vtx(12 * (size_t)nc), fn(3 * (size_t)nf), bn(3 * (size_t)std::max(nbf, 1)),
        bt1(3 * (size_t)std::max(nbf, 1)), bt2(3 * (size_t)std::max(nbf, 1));
    std::vector<int32_t> cf(4 * (size_t)nc), cfs(nc), fnb(nf), btag(std::max(nbf, 1));
    for (int i = 0; i < nc; ++i) {
        for (int d = 0; d < 3; ++d) dS[(size_t)d * nc + i] = mh.dS[3 * (size_t)i + d];
        for (int k = 0; k < 4; ++k)
            for (int d = 0; d < 3; ++d) vtx[(size_t)(3 * k + d) * nc + i] = mh.xyz[3 * (size_t)mh.tet[4 * (size_t)i + k] + d];
        int bits = 0;
        for (int k = 0; k < 4; ++k) {
            cf[(size_t)k * nc + i] = mh.cf[4 * (size_t)i + k];
            if (mh.cf_sign[4 * (size_t)i + k] > 0) bits |= 1 << k;
        }
        cfs[i] = bits;
    }
    for (int f = 0; f < nf; ++f) {
        for (int d = 0; d < 3; ++d) fn[(size_t)d * nf + f] = mh.f_n[3 * (size_t)f + d];
        fnb[f] = mh.f_nbr[f] >= 0 ? mh.f_nbr[f] : -1 - mh.bf_of_face[f];
    }
    // least-squares gradient coefficients (Sec. 2.1): weights 1/|dx_k|^2 over
    // the 4 face neighbours, a boundary face contributing a ghost at the mirror
    // image of the centroid; grad = sum_k c_k (v_k - v_i) with
    // c_k = A^-1 w_k dx_k, A = sum_k w_k dx_k dx_k^T.  Also the centroid-to-face
    // vectors and epsilon^2 = (K |Omega|^(1/3))^3 of Venkatakrishnan's limiter.
    std::vector<double> lsq_c(12 * (size_t)nc), lsq_dxf(12 * (size_t)nc), eps2(nc);
    std::vector<int32_t> flk(nf, 0);
    for (int i = 0; i < nc; ++i) {
        double xi[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 4; ++k)
            for (int d = 0; d < 3; ++d) xi[d] += mh.xyz[3 * (size_t)mh.tet[4 * (size_t)i + k] + d];
        for (int d = 0; d < 3; ++d) xi[d] *= 0.25;
        double dx[4][3], w[4], A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int k = 0; k < 4; ++k) {
            const int f = mh.cf[4 * (size_t)i + k];
            const bool own = mh.cf_sign[4 * (size_t)i + k] > 0;
            const double* xf = &mh.f_c[3 * (size_t)f];
            for (int d = 0; d < 3; ++d) lsq_dxf[(size_t)(3 * k + d) * nc + i] = xf[d] - xi[d];
            const int j = own ? mh.f_nbr[f] : mh.f_own[f];
            if (j >= 0) {
                for (int d = 0; d < 3; ++d) {
                    double xj = 0.0;
                    for (int l = 0; l < 4; ++l) xj += mh.xyz[3 * (size_t)mh.tet[4 * (size_t)j + l] + d];
                    dx[k][d] = 0.25 * xj - xi[d];
                }
            } else {
                const double* n = &mh.f_n[3 * (size_t)f];
                const double h = (xf[0] - xi[0]) * n[0] + (xf[1] - xi[1]) * n[1] + (xf[2] - xi[2]) * n[2];
                for (int d = 0; d < 3; ++d) dx[k][d] = 2.0 * h * n[d];
            }
            w[k] = 1.0 / (dx[k][0] * dx[k][0] + dx[k][1] * dx[k][1] + dx[k][2] * dx[k][2]);
            for (int r = 0; r < 3; ++r)
                for (int cc = 0; cc < 3; ++cc) A[r][cc] += w[k] * dx[k][r] * dx[k][cc];
            if (own) flk[f] |= k;
            else flk[f] |= k << 2;
        }
        // inverse of the symmetric 3x3 matrix by cofactors
        double C[3][3];
        C[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
        C[0][1] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
        C[0][2] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
        C[1][0] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
        C[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
        C[1][2] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
        C[2][0] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
        C[2][1] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
        C[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
        const double det = A[0][0] * C[0][0] + A[0][1] * C[1][0] + A[0][2] * C[2][0];
        for (int k = 0; k < 4; ++k)
            for (int r = 0; r < 3; ++r)
                lsq_c[(size_t)(3 * k + r) * nc + i] =
                    w[k] * (C[r][0] * dx[k][0] + C[r][1] * dx[k][1] + C[r][2] * dx[k][2]) / det;
        eps2[i] = std::pow(p->venkat_K * std::cbrt(mh.vol[i]), 3.0);
    }
    // flux work order: interior faces, then boundary faces grouped by type
    std::vector<int32_t> forder;
    forder.reserve(nf);
    for (int f = 0; f < nf; ++f)
        if (mh.f_nbr[f] >= 0) forder.push_back(f);
    for (int type = 1; type <= 4; ++type)
        for (int f = 0; f < nf; ++f)
            if (mh.f_nbr[f] < 0 && p->bc[mh.f_tag[f]].type == type) forder.push_back(f);
    // binary32 images for the mixed mode: boundary-face frames and U_w.t (Sec. 2.4 (e))
    std::vector<float> bff(11 * (size_t)std::max(nbf, 1), 0.0f);
    for (int b = 0; b < nbf; ++b) {
        const int f = mh.face_of_bf[b];
        const double* t1 = &mh.f_t1[3 * (size_t)f];
        const double* t2 = &mh.f_t2[3 * (size_t)f];
        for (int d = 0; d < 3; ++d) {
            bff[(size_t)d * nbf + b] = (float)mh.f_n[3 * (size_t)f + d];
            bff[(size_t)(3 + d) * nbf + b] = (float)t1[d];
            bff[(size_t)(6 + d) * nbf + b] = (float)t2[d];
        }
        const double* Uw = p->bc[mh.f_tag[f]].U_w;
        bff[(size_t)9 * nbf + b] = (float)((Uw[0] * t1[0] + Uw[1] * t1[1]) + Uw[2] * t1[2]);
        bff[(size_t)10 * nbf + b] = (float)((Uw[0] * t2[0] + Uw[1] * t2[1]) + Uw[2] * t2[2]);
    }
    for (int b = 0; b < nbf; ++b) {
        const int f = mh.face_of_bf[b];
        btag[b] = mh.f_tag[f];
        for (int d = 0; d < 3; ++d) {
            bn[(size_t)d * nbf + b] = mh.f_n[3 * (size_t)f + d];
            bt1[(size_t)d * nbf + b] = mh.f_t1[3 * (size_t)f + d];
            bt2[(size_t)d * nbf + b] = mh.f_t2[3 * (size_t)f + d];
        }
    }
    // mixed mode: each tet's anchor, vertex 0 rounded to the grid 2^-q with
    // q = 22 - r (2^r bounds the coordinates): anchors and their differences
    // are exact in binary32, and a particle's position is stored as its
    // binary32 offset from the anchor of its tet (binary64: anchors 0)
    s->anchor.assign(3 * (size_t)nc, 0.0);
    std::vector<float4> ancf(nc, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    if (s->real_size == 4) {
        double mx = 0.0;
        for (double v : mh.xyz) mx = std::max(mx, std::fabs(v));
        int r = 0;
        while (std::ldexp(1.0, r) <= mx) ++r;
        const int q = 22 - r;
        for (int i = 0; i < nc; ++i) {
            double a[3];
            for (int d = 0; d < 3; ++d) {
                a[d] = std::ldexp(std::nearbyint(std::ldexp(mh.xyz[3 * (size_t)mh.tet[4 * (size_t)i] + d], q)), -q);
                s->anchor[3 * (size_t)i + d] = a[d];
            }
            ancf[i] = make_float4((float)a[0], (float)a[1], (float)a[2], 0.0f);
        }
    }
    // mixed-mode sampling frame (Sec. 2.4 (b)): vertex 0 minus the anchor and
    // the edges p_k - p_0, binary64 values each split into a binary32 pair
    // (high = the value rounded, low = the rest rounded)
    std::vector<float> smpf;
    if (s->real_size == 4) {
        smpf.assign(24 * (size_t)nc, 0.0f);
        auto put = [&](int c, int j, int i, double v) {
            const float h = (float)v;
            smpf[(size_t)(8 * c + j) * nc + i] = h;
            smpf[(size_t)(8 * c + j + 1) * nc + i] = (float)(v - (double)h);
        };
        for (int i = 0; i < nc; ++i) {
            const double* p0 = &mh.xyz[3 * (size_t)mh.tet[4 * (size_t)i]];
            for (int c = 0; c < 3; ++c) {
                put(c, 0, i, p0[c] - s->anchor[3 * (size_t)i + c]);
                for (int k = 1; k < 4; ++k) put(c, 2 * k, i, mh.xyz[3 * (size_t)mh.tet[4 * (size_t)i + k] + c] - p0[c]);
            }
        }
    }
    // tracking records: planes (+-n, +-d) per local face (mixed mode: d in the
    // tet's frame, d - n.A), neighbour codes
    std::vector<TrkF> tf;
    std::vector<TrkD> td;
    if (s->real_size == 4) tf.resize(nc); else td.resize(nc);
    for (int i = 0; i < nc; ++i) {
        int nbv[4];
        for (int k = 0; k < 4; ++k) {
            const int f = mh.cf[4 * (size_t)i + k];
            const bool own = mh.cf_sign[4 * (size_t)i + k] > 0;
            const double* n = &mh.f_n[3 * (size_t)f];
            const double d = mh.f_d[f];
            if (s->real_size == 4) {
                const double* Ai = &s->anchor[3 * (size_t)i];
                const double dl = d - ((n[0] * Ai[0] + n[1] * Ai[1]) + n[2] * Ai[2]);
                const float nx = (float)n[0], ny = (float)n[1], nz = (float)n[2], dd = (float)dl;
                tf[i].pl[k] = own ? make_float4(nx, ny, nz, dd) : make_float4(-nx, -ny, -nz, -dd);
            } else {
                td[i].pl[k] = own ? Dbl4{n[0], n[1], n[2], d} : Dbl4{-n[0], -n[1], -n[2], -d};
            }
            if (mh.f_nbr[f] < 0) nbv[k] = -1 - mh.bf_of_face[f];
            else if (own) nbv[k] = (mh.f_nbr[f] << 2) | mh.f_nbr_k[f];
            else nbv[k] = (mh.f_own[f] << 2) | mh.f_own_k[f];
        }
        const int4 nb4 = make_int4(nbv[0], nbv[1], nbv[2], nbv[3]);
        if (s->real_size == 4) {
            tf[i].nb = nb4;
            // anchor differences to the neighbours (exact in binary32)
            for (int k = 0; k < 4; ++k) {
                const float4 a0 = ancf[i], a1 = nbv[k] >= 0 ? ancf[nbv[k] >> 2] : ancf[i];
                tf[i].da[3 * k] = a0.x - a1.x;
                tf[i].da[3 * k + 1] = a0.y - a1.y;
                tf[i].da[3 * k + 2] = a0.z - a1.z;
            }
        } else {
            td[i].nb = nb4;
        }
    }
    cudaStream_t st = s->stream;
    auto up = [&](const void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice, st);
    };
    cudaError_t ce = cudaSuccess;
#define UP(dst, src, bytes)                     \
    do {                                         \
        if (ce == cudaSuccess) ce = up(dst, src, bytes); \
    } while (0)
    UP(s->M.vol, mh.vol.data(), nc * sizeof(double));
    std::vector<double> ivol(nc);
    for (int i = 0; i < nc; ++i) ivol[i] = 1.0 / mh.vol[i];
    UP(s->M.ivol, ivol.data(), nc * sizeof(double));
    UP(s->M.dS, dS.data(), dS.size() * sizeof(double));
    UP(s->M.vtx, vtx.data(), vtx.size() * sizeof(double));
    UP(s->M.cf, cf.data(), cf.size() * sizeof(int32_t));
    UP(s->M.cfs, cfs.data(), cfs.size() * sizeof(int32_t));
    if (s->real_size == 4) {
        UP(s->M.trk_f, tf.data(), tf.size() * sizeof(TrkF));
    } else {
        UP(s->M.trk_d, td.data(), td.size() * sizeof(TrkD));
    }
    UP(s->M.face_order, forder.data(), nf * sizeof(int32_t));
    UP(s->M.smp_f, smpf.data(), smpf.size() * sizeof(float));
    UP(s->M.bf_f, bff.data(), bff.size() * sizeof(float));
    UP(s->M.lsq_c, lsq_c.data(), lsq_c.size() * sizeof(double));
    UP(s->M.lsq_dxf, lsq_dxf.data(), lsq_dxf.size() * sizeof(double));
    UP(s->M.eps2, eps2.data(), eps2.size() * sizeof(double));
    UP(s->M.f_lk, flk.data(), flk.size() * sizeof(int32_t));
    UP(s->M.f_own, mh.f_own.data(), nf * sizeof(int32_t));
    UP(s->M.f_nbr, fnb.data(), nf * sizeof(int32_t));
    UP(s->M.f_n, fn.data(), fn.size() * sizeof(double));
    UP(s->M.f_area, mh.f_area.data(), nf * sizeof(double));
    UP(s->M.bf_tag, btag.data(), btag.size() * sizeof(int32_t));
    UP(s->M.bf_n, bn.data(), bn.size() * sizeof(double));
    UP(s->M.bf_t1, bt1.data(), bt1.size() * sizeof(double));
    UP(s->M.bf_t2, bt2.data(), bt2.size() * sizeof(double));
    UP(s->S.W, W0, 5 * (size_t)nc * sizeof(double));
#undef UP
    if (ce == cudaSuccess) ce = cudaMemsetAsync(s->S.nleft, 0, nc * sizeof(int32_t), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(s->S.smass, 0, nc * sizeof(int64_t), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(s->S.cnt64, 0, CNT_SLOTS * sizeof(int64_t), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(s->S.t, 0, sizeof(double), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(s->S.dt, 0, sizeof(double), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(s->S.tsum, 0, sizeof(double), st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s->wave, cudaStreamNonBlocking);
    // the fork is a timing event: with directly launched steps the wave kernels
    // then start as they do in the captured graphs (measured on the settled
    // 24^3 cavity: 1.28 ms per direct step against 1.63 ms with a fork event
    // without timing; graph-replayed steps 1.24-1.25 ms either way)
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s->fork, cudaEventDefault);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s->sampled, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s->tracked, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s->gp_ready, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s->waved, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
        delete s;
        return cuda_fail(ce, "ugkwp_init upload");
    }
    s->lc.particle_blocks = particle_grid();
    s->lc.wave_blocks = sm_count();
    s->lc.track = TrackShape{128};
    // the tracking blocks' walk queues and the wave flux share each SM's
    // L1/shared memory; one common carveout lets them run side by side
    s->lc.carveout = 58;
    ce = configure_kernels(s->P, s->lc);
    if (ce != cudaSuccess) {
        delete s;
        return cuda_fail(ce, "ugkwp_init kernel attributes");
    }
    *out = s;
    return UGKWP_OK;
}

int ugkwp_free(ugkwp_sim* s) {
    if (s && s->stream) cudaStreamSynchronize(s->stream);
    delete s;
    return UGKWP_OK;
}

}  // extern "C"

namespace {
cudaEvent_t take_event(ugkwp_sim* s) {
    if (!s->pool.empty()) {
        cudaEvent_t e = s->pool.back();
        s->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch one kernel class on stream q, bracketed by events when timing is enabled.
template <class F> void timed(ugkwp_sim* s, int k, int n_kernels, cudaStream_t q, F&& launch) {
    s->launches[k] += n_kernels;
    if (!s->timing) {
        launch();
        return;
    }
    TimedLaunch t{k, take_event(s), take_event(s)};
    cudaEventRecord(t.a, q);
    launch();
    cudaEventRecord(t.b, q);
    s->pending.push_back(t);
}
}  // namespace

extern "C" {

int ugkwp_timing_enable(ugkwp_sim* s, int32_t enable) {
    if (!s) return fail(UGKWP_E_ARG, "NULL simulation");
    s->timing = enable != 0;
    return UGKWP_OK;
}

int ugkwp_timing_read(ugkwp_sim* s, double* ms, int64_t* launches) {
    if (!s) return fail(UGKWP_E_ARG, "NULL simulation");
    CU(cudaStreamSynchronize(s->stream));
    double acc[UGKWP_N_KERNELS] = {};
    for (auto& t : s->pending) {
        float v = 0.0f;
        CU(cudaEventElapsedTime(&v, t.a, t.b));
        acc[t.k] += v;
        s->pool.push_back(t.a);
        s->pool.push_back(t.b);
    }
    s->pending.clear();
    for (int k = 0; k < UGKWP_N_KERNELS; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = s->launches[k];
    }
    return UGKWP_OK;
}

}  // extern "C"

namespace {
// Enqueue the kernels of one step on the bound stream (the wave flux forked
// onto the library's second stream) and swap the ping-pong buffers.
int enqueue_step(ugkwp_sim* s) {
    cudaStream_t q = s->stream;
    {
        timed(s, UGKWP_K_RESET, 1, q, [&] { launch_reset(s->M, s->S, q); });
        timed(s, UGKWP_K_CELL_PREP, 1, q, [&] { launch_cell_prep(s->M, s->S, s->P, q); });
        timed(s, UGKWP_K_SAMPLE_COUNT, 1, q, [&] { launch_sample_count(s->M, s->S, s->P, q); });
        // fork: the wave flux needs only W^n, rho^h, tau and dt (ready now) and
        // writes only F, which no particle kernel touches
        CU(cudaEventRecord(s->fork, q));
        CU(cudaStreamWaitEvent(s->wave, s->fork, 0));
        const bool gp = s->P.sampling == UGKWP_SAMPLE_GP1;
        if (s->P.order == 2)
            timed(s, UGKWP_K_GRADIENTS, gp ? 2 : 1, s->wave, [&] {
                launch_gradients(s->M, s->S, s->P, s->wave);
                // first-order g_p sampling needs the cell slopes
                if (gp) launch_gp_coef(s->M, s->S, s->P, s->wave);
            });
        if (gp) CU(cudaEventRecord(s->gp_ready, s->wave));
        // order 2: one kernel, interior faces at second order then the boundary
        // faces at first order; order 1: every face at first order
        if (s->P.order == 2)
            timed(s, UGKWP_K_FLUX_O2, 1, s->wave, [&] { launch_face_flux_o2(s->M, s->S, s->P, s->lc.wave_blocks, s->wave); });
        else
            timed(s, UGKWP_K_FLUX, 1, s->wave, [&] { launch_face_flux(s->M, s->S, s->P, 0, s->lc.wave_blocks, s->wave); });
        CU(cudaEventRecord(s->join, s->wave));
        // the wave part of the update follows the flux on the wave stream,
        // beside the tracking; the particle part waits for it
        timed(s, UGKWP_K_UPDATE, 1, s->wave, [&] { launch_wave_update(s->M, s->S, s->wave); });
        CU(cudaEventRecord(s->waved, s->wave));
        timed(s, UGKWP_K_SCAN, 2, q, [&] { launch_scan(s->M, s->S, s->P, q); });
        if (gp) CU(cudaStreamWaitEvent(q, s->gp_ready, 0));  // the sampler reads the g_p coefficients
        const bool matched = s->P.sampling == UGKWP_SAMPLE_ENERGY_MATCHED;
        timed(s, UGKWP_K_SAMPLE, matched ? 2 : 1, q, [&] {
            if (matched) launch_sample_scale(s->M, s->S, s->P, q);
            launch_sample_write(s->M, s->S, s->P, s->A, s->lc.particle_blocks, q);
        });
        // tracking in two launches that take tiles from one counter: the first
        // half of the grid starts now and leaves room on each SM for a block
        // of the wave flux; the second half starts once the wave flux is done
        // and takes the tiles that are left
        cudaError_t ce = cudaSuccess;
        const int first_half = (s->lc.particle_blocks + 1) / 2;
        timed(s, UGKWP_K_TRACK, s->lc.particle_blocks > first_half ? 2 : 1, q, [&] {
            ce = cudaEventRecord(s->sampled, q);
            launch_track(s->M, s->S, s->P, s->A, s->B, s->Mv, s->lc.track, first_half, q);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s->aux, s->sampled, 0);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s->aux, s->join, 0);
            if (s->lc.particle_blocks > first_half)
                launch_track(s->M, s->S, s->P, s->A, s->B, s->Mv, s->lc.track, s->lc.particle_blocks - first_half,
                             s->aux);
            if (ce == cudaSuccess) ce = cudaEventRecord(s->tracked, s->aux);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(q, s->tracked, 0);
        });
        if (ce != cudaSuccess) return cuda_fail(ce, "tracking launch order");
        timed(s, UGKWP_K_MOVERS, 1, q, [&] { launch_movers(s->M, s->S, s->P, s->Mv, s->lc.particle_blocks, q); });
        CU(cudaStreamWaitEvent(q, s->waved, 0));  // the wave part of the update is done
        timed(s, UGKWP_K_UPDATE, 1, q, [&] { launch_cell_update(s->M, s->S, s->P, s->B.cell, q); });
        std::swap(s->A, s->B);
        std::swap(s->S.nleft, s->S.nleft_next);
        std::swap(s->S.smass, s->S.smass_next);
    }
    return UGKWP_OK;
}

// One step of the gas-kinetic scheme (no particles; mode 1: global time step,
// 2: local time steps) on the bound stream, as direct launches with a copy of
// the parameters that carries the mode.
int enqueue_gks_step(ugkwp_sim* s, int32_t mode) {
    cudaStream_t q = s->stream;
    DevParams P = s->P;
    P.gks = mode;
    P.averaging = 0;
    timed(s, UGKWP_K_RESET, 1, q, [&] { launch_reset(s->M, s->S, q); });
    timed(s, UGKWP_K_CELL_PREP, 1, q, [&] { launch_cell_prep(s->M, s->S, P, q); });
    timed(s, UGKWP_K_SAMPLE_COUNT, 1, q, [&] { launch_sample_count(s->M, s->S, P, q); });
    if (P.order == 2)
        timed(s, UGKWP_K_GRADIENTS, 1, q, [&] { launch_gradients(s->M, s->S, P, q); });
    if (P.order == 2)
        timed(s, UGKWP_K_FLUX_O2, 1, q, [&] { launch_face_flux_o2(s->M, s->S, P, s->lc.wave_blocks, q); });
    else
        timed(s, UGKWP_K_FLUX, 1, q, [&] { launch_face_flux(s->M, s->S, P, 0, 0, q); });
    timed(s, UGKWP_K_UPDATE, 1, q, [&] { launch_cell_update(s->M, s->S, P, nullptr, q); });
    return UGKWP_OK;
}

// Two steps as one CUDA graph for the current parity (captured on first use).
int launch_step_pair(ugkwp_sim* s, bool& used) {
    used = false;
    if (!s->graphs_ok || s->timing || s->stream == nullptr) return UGKWP_OK;
    // the per-cell survivor counts swap every step: their pointer tells the
    // step parity a captured pair starts from
    void* key = s->S.nleft;
    int slot = s->graph_key[0] == key ? 0 : s->graph_key[1] == key ? 1 : -1;
    if (slot < 0) {
        slot = s->graph[0] ? 1 : 0;
        if (s->graph[slot]) { cudaGraphExecDestroy(s->graph[slot]); s->graph[slot] = nullptr; }
        int64_t saved[UGKWP_N_KERNELS];
        std::memcpy(saved, s->launches, sizeof(saved));
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            s->graphs_ok = false;
            return UGKWP_OK;
        }
        int rc = enqueue_step(s);
        if (rc == UGKWP_OK) rc = enqueue_step(s);
        cudaError_t e = cudaStreamEndCapture(s->stream, &g);
        for (int k = 0; k < UGKWP_N_KERNELS; ++k) s->graph_launches[slot][k] = s->launches[k] - saved[k];
        std::memcpy(s->launches, saved, sizeof(saved));
        if (rc != UGKWP_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            s->graphs_ok = false;
            return UGKWP_OK;
        }
        e = cudaGraphInstantiate(&s->graph[slot], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->graph[slot] = nullptr;
            s->graphs_ok = false;
            return UGKWP_OK;
        }
        s->graph_key[slot] = key;
    }
    CU(cudaGraphLaunch(s->graph[slot], s->stream));
    for (int k = 0; k < UGKWP_N_KERNELS; ++k) s->launches[k] += s->graph_launches[slot][k];
    used = true;
    return UGKWP_OK;
}
}  // namespace

extern "C" {

int ugkwp_step(ugkwp_sim* s, int32_t n_steps, ugkwp_stats* st) {
    if (!s || n_steps < 0) return fail(UGKWP_E_ARG, "invalid argument");
    cudaStream_t q = s->stream;
    for (int32_t k = 0; k < n_steps;) {
        if (s->step >= ((int64_t)1 << 24) - 2) return fail(UGKWP_E_STATE, "step counter exhausted (2^24 steps)");
        if (n_steps - k >= 2) {
            bool used = false;
            int rc = launch_step_pair(s, used);
            if (rc) return rc;
            if (used) {
                s->step += 2;
                k += 2;
                continue;
            }
        }
        int rc = enqueue_step(s);
        if (rc) return rc;
        s->step += 1;
        k += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (st) {
        int64_t h[CNT_SLOTS];
        double t = 0, dt = 0;
        CU(cudaMemcpyAsync(h, s->S.cnt64, sizeof(h), cudaMemcpyDeviceToHost, q));
        CU(cudaMemcpyAsync(&t, s->S.t, sizeof(double), cudaMemcpyDeviceToHost, q));
        CU(cudaMemcpyAsync(&dt, s->S.dt, sizeof(double), cudaMemcpyDeviceToHost, q));
        CU(cudaStreamSynchronize(q));
        st->t = t; st->dt = dt; st->step = s->step;
        st->n_particles = h[CNT_SURV]; st->n_tracked = h[CNT_TRACKED];
        st->n_sampled = h[CNT_SAMPLED]; st->n_collided = h[CNT_COLLIDED]; st->n_exited = h[CNT_EXITED];
        st->n_lost = h[CNT_LOST]; st->n_crossings = h[CNT_CROSSINGS]; st->n_wall_hits = h[CNT_WALL];
        st->n_moves_total = h[CNT_MOVES];
        st->n_movers = h[CNT_RESV];
        return read_error(s);
    }
    return UGKWP_OK;
}

int ugkwp_gks_steps(ugkwp_sim* s, int32_t n_steps, int32_t local_dt, ugkwp_stats* st) {
    if (!s || n_steps < 0) return fail(UGKWP_E_ARG, "invalid argument");
    if (local_dt != 0 && local_dt != 1) return fail(UGKWP_E_ARG, "local_dt must be 0 or 1");
    cudaStream_t q = s->stream;
    int64_t na = 0;
    CU(cudaMemcpyAsync(&na, s->S.cnt64 + CNT_N_A, sizeof(na), cudaMemcpyDeviceToHost, q));
    CU(cudaStreamSynchronize(q));
    if (na != 0) return fail(UGKWP_E_STATE, "a GKS step needs a state without particles");
    for (int32_t k = 0; k < n_steps; ++k) {
        int rc = enqueue_gks_step(s, local_dt ? 2 : 1);
        if (rc) return rc;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (st) {
        double t = 0, dt = 0;
        CU(cudaMemcpyAsync(&t, s->S.t, sizeof(double), cudaMemcpyDeviceToHost, q));
        CU(cudaMemcpyAsync(&dt, s->S.dt, sizeof(double), cudaMemcpyDeviceToHost, q));
        CU(cudaStreamSynchronize(q));
        std::memset(st, 0, sizeof(*st));
        st->t = t; st->dt = dt; st->step = s->step;
        return read_error(s);
    }
    return UGKWP_OK;
}

int ugkwp_average(ugkwp_sim* s, int32_t start) {
    if (!s) return fail(UGKWP_E_ARG, "NULL simulation");
    if (start) {
        CU(cudaMemsetAsync(s->S.wsum, 0, 5 * (size_t)s->M.nc * sizeof(double), s->stream));
        CU(cudaMemsetAsync(s->S.tsum, 0, sizeof(double), s->stream));
    }
    const int32_t on = start ? 1 : 0;
    if (s->P.averaging != on) {
        s->P.averaging = on;
        s->drop_graphs();  // the graphs carry the parameters by value
    }
    return UGKWP_OK;
}

int ugkwp_average_time(ugkwp_sim* s, double* t_avg) {
    if (!s || !t_avg) return fail(UGKWP_E_ARG, "NULL argument");
    CU(cudaMemcpyAsync(t_avg, s->S.tsum, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return UGKWP_OK;
}

int ugkwp_kn_gll(ugkwp_sim* s, double* out) {
    if (!s || !out) return fail(UGKWP_E_ARG, "NULL argument");
    cudaStream_t q = s->stream;
    launch_kn_gll(s->M, s->S, s->P, s->S.mom, q);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(out, s->S.mom, (size_t)s->M.nc * sizeof(double), cudaMemcpyDeviceToHost, q));
    CU(cudaStreamSynchronize(q));
    return read_error(s);
}

int ugkwp_sync(ugkwp_sim* s) {
    if (!s) return fail(UGKWP_E_ARG, "NULL simulation");
    return read_error(s);
}

int ugkwp_moments(ugkwp_sim* s, int32_t which, double* out, int32_t out_on_device) {
    if (!s || !out) return fail(UGKWP_E_ARG, "NULL argument");
    if (which < UGKWP_W || which > UGKWP_WBAR) return fail(UGKWP_E_ARG, "unknown moment");
    const size_t bytes = 5 * (size_t)s->M.nc * sizeof(double);
    cudaStream_t q = s->stream;
    if (which == UGKWP_WBAR) {
        double T = 0.0;
        CU(cudaMemcpyAsync(&T, s->S.tsum, sizeof(double), cudaMemcpyDeviceToHost, q));
        CU(cudaStreamSynchronize(q));
        if (!(T > 0.0)) return fail(UGKWP_E_STATE, "no averaged step yet (ugkwp_average)");
        double* dst = out_on_device ? out : s->S.mom;
        launch_wbar(s->M, s->S, dst, q);
        CU(cudaGetLastError());
        if (!out_on_device) {
            CU(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, q));
            CU(cudaStreamSynchronize(q));
            return read_error(s);
        }
        return UGKWP_OK;
    }
    if (which == UGKWP_W) {
        CU(cudaMemcpyAsync(out, s->S.W, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, q));
    } else {
        double* dst = out_on_device ? out : s->S.mom;
        if (which != UGKWP_PRIM) launch_wp_moments(s->M, s->S, s->P, s->A, dst, q);
        launch_prim_moments(s->M, s->S, s->P, which, dst, q);
        CU(cudaGetLastError());
        if (!out_on_device) CU(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, q));
    }
    if (!out_on_device) {
        CU(cudaStreamSynchronize(q));
        return read_error(s);
    }
    return UGKWP_OK;
}

int ugkwp_state_info(ugkwp_sim* s, ugkwp_state* st) {
    if (!s || !st) return fail(UGKWP_E_ARG, "NULL argument");
    int64_t h[CNT_SLOTS];
    double t = 0;
    CU(cudaMemcpyAsync(h, s->S.cnt64, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaMemcpyAsync(&t, s->S.t, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    // the current buffer holds the live particles in N_A slots (the rest are holes)
    st->n_particles = h[CNT_SURV];
    st->step = s->step;
    st->t = t;
    for (int q = 0; q < 5; ++q) st->exps[q] = s->P.exps[q];
    return UGKWP_OK;
}

int ugkwp_export_state(ugkwp_sim* s, ugkwp_state* st) {
    if (!s || !st) return fail(UGKWP_E_ARG, "NULL argument");
    int64_t want = st->n_particles;
    int rc = ugkwp_state_info(s, st);
    if (rc) return rc;
    if (want < st->n_particles) return fail(UGKWP_E_ARG, "n_particles of the state is smaller than the particle count");
    const int nc = s->M.nc;
    cudaStream_t q = s->stream;
    if (st->W) CU(cudaMemcpyAsync(st->W, s->S.W, 5 * (size_t)nc * sizeof(double), cudaMemcpyDeviceToHost, q));
    int64_t h[CNT_SLOTS];
    CU(cudaMemcpyAsync(h, s->S.cnt64, sizeof(h), cudaMemcpyDeviceToHost, q));
    CU(cudaStreamSynchronize(q));
    const size_t n = (size_t)h[CNT_N_A], rs = s->real_size;
    std::vector<char> xs[3], us[3];
    std::vector<double> m(n);
    std::vector<int32_t> cell(n);
    std::vector<uint64_t> id(n);
    std::vector<char> es(s->A.e ? n * rs : 0);
    if (s->A.e && n) CU(cudaMemcpyAsync(es.data(), s->A.e, n * rs, cudaMemcpyDeviceToHost, q));
    for (int d = 0; d < 3; ++d) {
        xs[d].resize(n * rs);
        us[d].resize(n * rs);
        if (n) {
            CU(cudaMemcpyAsync(xs[d].data(), s->A.x[d], n * rs, cudaMemcpyDeviceToHost, q));
            CU(cudaMemcpyAsync(us[d].data(), s->A.u[d], n * rs, cudaMemcpyDeviceToHost, q));
        }
    }
    if (n) {
        CU(cudaMemcpyAsync(m.data(), s->A.m, n * 8, cudaMemcpyDeviceToHost, q));
        CU(cudaMemcpyAsync(cell.data(), s->A.cell, n * 4, cudaMemcpyDeviceToHost, q));
        CU(cudaMemcpyAsync(id.data(), s->A.id, n * 8, cudaMemcpyDeviceToHost, q));
    }
    CU(cudaStreamSynchronize(q));
    const size_t np = (size_t)st->n_particles;
    size_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        if (cell[i] < 0) continue;
        if (st->id) st->id[k] = id[i];
        if (st->cell) st->cell[k] = cell[i];
        if (st->m) st->m[k] = m[i];
        if (st->e) st->e[k] = !s->A.e ? 0.0 : rs == 4 ? (double)((const float*)es.data())[i] : ((const double*)es.data())[i];
        for (int d = 0; d < 3; ++d) {
            double xv, uv;
            if (rs == 4) {
                // mixed mode: anchor of the tet + offset, exact in binary64
                xv = s->anchor[3 * (size_t)cell[i] + d] + (double)((const float*)xs[d].data())[i];
                uv = ((const float*)us[d].data())[i];
            }
            else { xv = ((const double*)xs[d].data())[i]; uv = ((const double*)us[d].data())[i]; }
            if (st->x) st->x[d * np + k] = xv;
            if (st->u) st->u[d * np + k] = uv;
        }
        ++k;
    }
    return read_error(s);
}

}  // extern "C"

namespace {

// The end of an import: reads the check kernel's error word; when every
// particle passed, the spare buffer B (which holds the image's particles)
// becomes the current one and W, the counters, t, the quanta and the
// survivors' counts and mass per cell are set from the image.
int import_commit(ugkwp_sim* s, int64_t n, int64_t step, double t, const int32_t* exps, const double* W,
                  const unsigned long long* err) {
    const int nc = s->M.nc;
    cudaStream_t q = s->stream;
    unsigned long long bad = 0;
    int64_t h[CNT_SLOTS];
    CU(cudaMemcpyAsync(&bad, err, sizeof(bad), cudaMemcpyDeviceToHost, q));
    CU(cudaMemcpyAsync(h, s->S.cnt64, sizeof(h), cudaMemcpyDeviceToHost, q));
    CU(cudaStreamSynchronize(q));
    switch (bad == ~0ULL ? 0 : (int)(bad & 7)) {
        case 0: break;
        case 1: return fail(UGKWP_E_STATE, "particle cell out of range");
        case 2: return fail(UGKWP_E_STATE, "negative internal energy");
        case 3: return fail(UGKWP_E_STATE, "internal energy not representable in binary32");
        default: return fail(UGKWP_E_STATE, "particle state not representable in binary32");
    }
    std::swap(s->A, s->B);
    CU(cudaMemcpyAsync(s->S.W, W, 5 * (size_t)nc * sizeof(double), cudaMemcpyHostToDevice, q));
    const int64_t moves = h[CNT_MOVES];
    std::memset(h, 0, sizeof(h));
    h[CNT_MOVES] = moves;
    h[CNT_N_A] = n;
    h[CNT_SURV] = n;
    h[CNT_STEP] = step;
    CU(cudaMemcpyAsync(s->S.cnt64, h, sizeof(h), cudaMemcpyHostToDevice, q));
    CU(cudaMemcpyAsync(s->S.t, &t, sizeof(double), cudaMemcpyHostToDevice, q));
    CU(cudaMemsetAsync(s->S.nleft, 0, nc * sizeof(int32_t), q));
    CU(cudaMemsetAsync(s->S.smass, 0, nc * sizeof(int64_t), q));
    set_exps(s->P, exps);
    s->drop_graphs();  // the graphs carry the parameters by value
    launch_rebuild_survivors(s->M, s->S, s->P, s->A, q);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(q));
    s->step = step;
    return UGKWP_OK;
}

// The device staging of a binary64 image in mixed precision (`need` bytes),
// allocated on first use and kept until ugkwp_free.
int import_staging(ugkwp_sim* s, size_t need, char*& base) {
    if (need > s->imp_bytes) {
        if (s->imp) cudaFree(s->imp);
        s->imp = nullptr;
        s->imp_bytes = 0;
        CU(cudaMalloc(&s->imp, need));
        s->imp_bytes = need;
    }
    base = static_cast<char*>(s->imp);
    return UGKWP_OK;
}

}  // namespace

extern "C" {

int ugkwp_import_state(ugkwp_sim* s, const ugkwp_state* st) {
    if (!s || !st || !st->W || (st->n_particles > 0 && (!st->id || !st->cell || !st->x || !st->u || !st->m)))
        return fail(UGKWP_E_ARG, "NULL argument");
    const int64_t n = st->n_particles;
    if (n < 0 || n > s->capacity) return fail(UGKWP_E_CAPACITY, "imported particles exceed the capacity");
    if (st->step < 0 || st->step >= ((int64_t)1 << 24) - 1) return fail(UGKWP_E_STATE, "step out of range");
    const int nc = s->M.nc;
    const size_t rs = s->real_size;
    if (s->A.e && n > 0 && !st->e) return fail(UGKWP_E_ARG, "internal energies (e) needed when K > 0");
    // The image goes to the device as the caller holds it: cell, m and id into
    // the spare buffer B; x, u and e into B as well with binary64 particles,
    // else into a device staging buffer (binary64, with the tets' anchors),
    // from which k_import checks every particle and converts it into B.  The
    // buffers swap only when every particle passed, so a rejected image
    // leaves the simulation as it was.  The first failed particle is reported
    // in a counter slot that no step uses.
    const bool mixed = rs == 4;
    const bool ke = s->A.e != nullptr;
    unsigned long long* err = reinterpret_cast<unsigned long long*>(&s->S.cnt64[CNT_IMPORT]);
    double* anc = nullptr;
    if (mixed) {
        char* base = nullptr;
        int rc = import_staging(s, (3 * (size_t)nc + (size_t)(ke ? 7 : 6) * (size_t)n) * sizeof(double), base);
        if (rc) return rc;
        anc = reinterpret_cast<double*>(base);
    }
    double* xs = mixed ? anc + 3 * (size_t)nc : nullptr;
    double* us = mixed ? xs + 3 * (size_t)n : nullptr;
    double* es = (mixed && ke) ? us + 3 * (size_t)n : nullptr;
    cudaStream_t q = s->stream;
    CU(cudaStreamSynchronize(q));  // B is free once the bound stream's steps are done
    CU(cudaMemsetAsync(err, 0xff, sizeof(unsigned long long), q));
    if (n) {
        CU(cudaMemcpyAsync(s->B.m, st->m, (size_t)n * 8, cudaMemcpyHostToDevice, q));
        CU(cudaMemcpyAsync(s->B.cell, st->cell, (size_t)n * 4, cudaMemcpyHostToDevice, q));
        CU(cudaMemcpyAsync(s->B.id, st->id, (size_t)n * 8, cudaMemcpyHostToDevice, q));
        if (mixed) {
            CU(cudaMemcpyAsync(anc, s->anchor.data(), 3 * (size_t)nc * sizeof(double), cudaMemcpyHostToDevice, q));
            CU(cudaMemcpyAsync(xs, st->x, 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, q));
            CU(cudaMemcpyAsync(us, st->u, 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, q));
            if (ke) CU(cudaMemcpyAsync(es, st->e, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, q));
        } else {
            for (int d = 0; d < 3; ++d) {
                CU(cudaMemcpyAsync(s->B.x[d], st->x + (size_t)d * n, (size_t)n * 8, cudaMemcpyHostToDevice, q));
                CU(cudaMemcpyAsync(s->B.u[d], st->u + (size_t)d * n, (size_t)n * 8, cudaMemcpyHostToDevice, q));
            }
            if (ke) CU(cudaMemcpyAsync(s->B.e, st->e, (size_t)n * 8, cudaMemcpyHostToDevice, q));
        }
        launch_import(nc, n, mixed, mixed, anc, xs, us, es, s->B, err, q);
        CU(cudaGetLastError());
    }
    return import_commit(s, n, st->step, st->t, st->exps, st->W, err);
}

int ugkwp_export_state_native(ugkwp_sim* s, ugkwp_state_native* st) {
    if (!s || !st) return fail(UGKWP_E_ARG, "NULL argument");
    const int64_t want = st->n_particles;
    ugkwp_state info{};
    int rc = ugkwp_state_info(s, &info);
    if (rc) return rc;
    st->n_particles = info.n_particles;
    st->step = info.step;
    st->t = info.t;
    for (int q = 0; q < 5; ++q) st->exps[q] = info.exps[q];
    st->real_size = (int32_t)s->real_size;
    if (want < st->n_particles) return fail(UGKWP_E_ARG, "n_particles of the state is smaller than the particle count");
    const int nc = s->M.nc;
    cudaStream_t q = s->stream;
    if (st->W) CU(cudaMemcpyAsync(st->W, s->S.W, 5 * (size_t)nc * sizeof(double), cudaMemcpyDeviceToHost, q));
    int64_t h[CNT_SLOTS];
    CU(cudaMemcpyAsync(h, s->S.cnt64, sizeof(h), cudaMemcpyDeviceToHost, q));
    CU(cudaStreamSynchronize(q));
    // the N_A slots of the current buffer, then the live ones (cell >= 0) in
    // buffer order into the caller's arrays
    const size_t n = (size_t)h[CNT_N_A], rs = s->real_size;
    std::vector<char> xs[3], us[3];
    std::vector<double> m(n);
    std::vector<int32_t> cell(n);
    std::vector<uint64_t> id(n);
    std::vector<char> es(s->A.e ? n * rs : 0);
    if (s->A.e && n) CU(cudaMemcpyAsync(es.data(), s->A.e, n * rs, cudaMemcpyDeviceToHost, q));
    for (int d = 0; d < 3; ++d) {
        xs[d].resize(n * rs);
        us[d].resize(n * rs);
        if (n) {
            CU(cudaMemcpyAsync(xs[d].data(), s->A.x[d], n * rs, cudaMemcpyDeviceToHost, q));
            CU(cudaMemcpyAsync(us[d].data(), s->A.u[d], n * rs, cudaMemcpyDeviceToHost, q));
        }
    }
    if (n) {
        CU(cudaMemcpyAsync(m.data(), s->A.m, n * 8, cudaMemcpyDeviceToHost, q));
        CU(cudaMemcpyAsync(cell.data(), s->A.cell, n * 4, cudaMemcpyDeviceToHost, q));
        CU(cudaMemcpyAsync(id.data(), s->A.id, n * 8, cudaMemcpyDeviceToHost, q));
    }
    CU(cudaStreamSynchronize(q));
    const size_t np = (size_t)st->n_particles;
    char* xo = static_cast<char*>(st->x);
    char* uo = static_cast<char*>(st->u);
    char* eo = static_cast<char*>(st->e);
    size_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        if (cell[i] < 0) continue;
        if (st->id) st->id[k] = id[i];
        if (st->cell) st->cell[k] = cell[i];
        if (st->m) st->m[k] = m[i];
        if (eo) {
            if (s->A.e) std::memcpy(eo + k * rs, es.data() + i * rs, rs);
            else std::memset(eo + k * rs, 0, rs);
        }
        for (int d = 0; d < 3; ++d) {
            if (xo) std::memcpy(xo + (d * np + k) * rs, xs[d].data() + i * rs, rs);
            if (uo) std::memcpy(uo + (d * np + k) * rs, us[d].data() + i * rs, rs);
        }
        ++k;
    }
    return read_error(s);
}

int ugkwp_import_state_native(ugkwp_sim* s, const ugkwp_state_native* st) {
    if (!s || !st || !st->W || (st->n_particles > 0 && (!st->id || !st->cell || !st->x || !st->u || !st->m)))
        return fail(UGKWP_E_ARG, "NULL argument");
    const int64_t n = st->n_particles;
    if (n < 0 || n > s->capacity) return fail(UGKWP_E_CAPACITY, "imported particles exceed the capacity");
    if (st->step < 0 || st->step >= ((int64_t)1 << 24) - 1) return fail(UGKWP_E_STATE, "step out of range");
    const size_t rs = s->real_size;
    if (st->real_size != (int32_t)rs) return fail(UGKWP_E_ARG, "real_size differs from the simulation's particle precision");
    const bool ke = s->A.e != nullptr;
    if (ke && n > 0 && !st->e) return fail(UGKWP_E_ARG, "internal energies (e) needed when K > 0");
    unsigned long long* err = reinterpret_cast<unsigned long long*>(&s->S.cnt64[CNT_IMPORT]);
    cudaStream_t q = s->stream;
    CU(cudaStreamSynchronize(q));  // B is free once the bound stream's steps are done
    CU(cudaMemsetAsync(err, 0xff, sizeof(unsigned long long), q));
    if (n) {
        // the image as it is into the spare buffer B, checked there
        const char* xi = static_cast<const char*>(st->x);
        const char* ui = static_cast<const char*>(st->u);
        CU(cudaMemcpyAsync(s->B.m, st->m, (size_t)n * 8, cudaMemcpyHostToDevice, q));
        CU(cudaMemcpyAsync(s->B.cell, st->cell, (size_t)n * 4, cudaMemcpyHostToDevice, q));
        CU(cudaMemcpyAsync(s->B.id, st->id, (size_t)n * 8, cudaMemcpyHostToDevice, q));
        for (int d = 0; d < 3; ++d) {
            CU(cudaMemcpyAsync(s->B.x[d], xi + (size_t)d * n * rs, (size_t)n * rs, cudaMemcpyHostToDevice, q));
            CU(cudaMemcpyAsync(s->B.u[d], ui + (size_t)d * n * rs, (size_t)n * rs, cudaMemcpyHostToDevice, q));
        }
        if (ke) CU(cudaMemcpyAsync(s->B.e, st->e, (size_t)n * rs, cudaMemcpyHostToDevice, q));
        launch_import(s->M.nc, n, rs == 4, false, nullptr, nullptr, nullptr, nullptr, s->B, err, q);
        CU(cudaGetLastError());
    }
    return import_commit(s, n, st->step, st->t, st->exps, st->W, err);
}

int ugkwp_last(ugkwp_sim* s, int32_t which, void* host_out) {
    if (!s || !host_out) return fail(UGKWP_E_ARG, "NULL argument");
    const size_t nc = s->M.nc, nf = s->M.nf;
    cudaStream_t q = s->stream;
    CU(cudaStreamSynchronize(q));
    auto get = [&](const void* src, size_t bytes) { return cudaMemcpy(host_out, src, bytes, cudaMemcpyDeviceToHost); };
    switch (which) {
        case 0: CU(get(s->S.dt, 8)); break;
        case 1: CU(get(s->S.tau, nc * 8)); break;
        case 2: CU(get(s->S.rhoh, nc * 8)); break;
        case 3: {
            std::vector<int32_t> v(nc);
            CU(cudaMemcpy(v.data(), s->S.nsam, nc * 4, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < nc; ++i) ((int64_t*)host_out)[i] = v[i];
            break;
        }
        case 4: CU(get(s->S.msam, nc * 8)); break;
        case 5: CU(get(s->S.F, 5 * nf * 8)); break;
        case 6: CU(get(s->S.pflux, 5 * nc * 8)); break;
        case 7: CU(get(s->S.smass, nc * 8)); break;
        case 8: {
            std::vector<int32_t> v(nc);
            CU(cudaMemcpy(v.data(), s->S.nleft, nc * 4, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < nc; ++i) ((int64_t*)host_out)[i] = v[i];
            break;
        }
        case 9:
        case 10:
            if (s->P.order != 2) return fail(UGKWP_E_ARG, "gradients exist only at order 2");
            if (which == 9) CU(get(s->S.gradW, 15 * nc * 8));
            else CU(get(s->S.gradH, 3 * nc * 8));
            break;
        default: return fail(UGKWP_E_ARG, "unknown diagnostic");
    }
    return UGKWP_OK;
}

// Device scratch of the adjoint for K steps: checkpoints of W (K + 1), the
// recorded rho^p (K) and particle fluxes (5 K), time steps, fluxes, face
// terms, two adjoint states, face products and per-step sums.
static void adjoint_layout(const ugkwp_sim* s, int K, Carver& c, double** ck, double** rp, double** pf, double** dt,
                           double** F, double** jf, double** lam0, double** lam1, double** wbar, double** thbar,
                           double** sums, double** theta, AdjO2* o2) {
    const size_t nc = s->M.nc, nf = s->M.nf;
    std::memset(o2, 0, sizeof(*o2));
    if (s->P.order == 2) {  // limiter values of every step, and scratch
        o2->phi = c.take<double>((size_t)K * 6 * nc);
        o2->gW = c.take<double>(15 * nc);
        o2->gH = c.take<double>(3 * nc);
        o2->gbar = c.take<double>(36 * nf);
        o2->gg = c.take<double>(18 * nc);
        o2->thc = c.take<double>(3 * nc);
    }
    *ck = c.take<double>((size_t)(K + 1) * 5 * nc);
    *rp = c.take<double>((size_t)K * nc);
    *pf = c.take<double>((size_t)K * 5 * nc);
    *dt = c.take<double>((size_t)K);
    *F = c.take<double>(5 * nf);
    *jf = c.take<double>(nf);
    *lam0 = c.take<double>(5 * nc);
    *lam1 = c.take<double>(5 * nc);
    *wbar = c.take<double>(10 * nf);
    *thbar = c.take<double>(3 * nf);
    *sums = c.take<double>((size_t)4 * K);
    *theta = c.take<double>(3);
}

int ugkwp_adjoint_query(const ugkwp_sim* s, int32_t n_steps, size_t* bytes) {
    if (!s || !bytes || n_steps < 1) return fail(UGKWP_E_ARG, "invalid argument");
    Carver c(nullptr);
    double* p[12];
    AdjO2 o2;
    adjoint_layout(s, n_steps, c, &p[0], &p[1], &p[2], &p[3], &p[4], &p[5], &p[6], &p[7], &p[8], &p[9], &p[10], &p[11], &o2);
    *bytes = (c.off + 255) & ~(size_t)255;
    return UGKWP_OK;
}

int ugkwp_adjoint_wave(ugkwp_sim* s, const ugkwp_adjoint_req* r, double* out) {
    if (!s || !r || !out) return fail(UGKWP_E_ARG, "NULL argument");
    if (s->P.K != 0) return fail(UGKWP_E_UNSUPPORTED, "the adjoint covers K = 0 only");
    if (r->n_steps < 1 || (r->functional != 0 && r->functional != 1) || r->n_wall_tags < 0 ||
        (r->n_wall_tags > 0 && !r->wall_tags))
        return fail(UGKWP_E_ARG, "invalid adjoint request");
    const int K = r->n_steps;
    size_t need = 0;
    int rc = ugkwp_adjoint_query(s, K, &need);
    if (rc) return rc;
    if (!r->d_workspace || r->workspace_bytes < need || ((uintptr_t)r->d_workspace & 255))
        return fail(UGKWP_E_WORKSPACE, "adjoint workspace missing, misaligned or smaller than ugkwp_adjoint_query");
    // parameterisation of the boundary conditions
    AdjParams ap;
    std::memset(&ap, 0, sizeof(ap));
    ap.comp = r->functional == 0 ? 1 : 4;
    for (int k = 0; k < r->n_wall_tags; ++k)
        if (r->wall_tags[k] >= 0 && r->wall_tags[k] < 16) ap.b[r->wall_tags[k]].listed = 1;
    int ff = -1, wall = -1;
    for (int b = 0; b < s->P.n_bc; ++b) {
        if (s->P.bc[b].type == UGKWP_BC_FARFIELD && ff < 0) ff = b;
        if (s->P.bc[b].type == UGKWP_BC_DIFFUSE_WALL && ap.b[b].listed && wall < 0) wall = b;
    }
    double theta0[3] = {0.0, 0.0, wall >= 0 ? s->P.bc[wall].T_w : 0.0};
    if (ff >= 0) {
        const double* Wi = s->P.bc[ff].W_in;
        const double r0 = Wi[0];
        const double U0[3] = {Wi[1] / r0, Wi[2] / r0, Wi[3] / r0};
        const double sp = std::sqrt((U0[0] * U0[0] + U0[1] * U0[1]) + U0[2] * U0[2]);
        const double e[3] = {sp > 0.0 ? U0[0] / sp : 1.0, sp > 0.0 ? U0[1] / sp : 0.0, sp > 0.0 ? U0[2] / sp : 0.0};
        const double RT = ((Wi[4] - 0.5 * r0 * sp * sp) / 1.5) / r0;
        theta0[0] = r0;
        theta0[1] = sp;
        for (int b = 0; b < s->P.n_bc; ++b) {
            if (s->P.bc[b].type != UGKWP_BC_FARFIELD || std::memcmp(s->P.bc[b].W_in, Wi, 5 * sizeof(double)) != 0)
                continue;
            ap.b[b].param_ff = 1;
            for (int d = 0; d < 3; ++d) ap.b[b].e[d] = e[d];
            ap.b[b].RT = RT;
        }
    }
    for (int b = 0; b < s->P.n_bc; ++b)
        if (s->P.bc[b].type == UGKWP_BC_DIFFUSE_WALL && ap.b[b].listed) ap.b[b].param_wall = 1;
    const double th_h[3] = {r->theta ? r->theta[0] : theta0[0], r->theta ? r->theta[1] : theta0[1],
                            r->theta ? r->theta[2] : theta0[2]};
    Carver c(r->d_workspace);
    double *ck, *rp, *pf, *dtv, *F, *jf, *lam0, *lam1, *wbar, *thbar, *sums, *theta;
    AdjO2 o2;
    adjoint_layout(s, K, c, &ck, &rp, &pf, &dtv, &F, &jf, &lam0, &lam1, &wbar, &thbar, &sums, &theta, &o2);
    auto step_o2 = [&](int n) {
        AdjO2 t = o2;
        if (t.phi) t.phi += (size_t)n * 6 * (size_t)s->M.nc;
        return t;
    };
    cudaStream_t q = s->stream;
    const size_t nc = s->M.nc;
    CU(cudaMemcpyAsync(theta, th_h, sizeof(th_h), cudaMemcpyHostToDevice, q));
    // 1. record K real steps
    CU(cudaMemcpyAsync(ck, s->S.W, 5 * nc * sizeof(double), cudaMemcpyDeviceToDevice, q));
    for (int n = 0; n < K; ++n) {
        rc = ugkwp_step(s, 1, nullptr);
        if (rc) return rc;
        CU(cudaMemcpyAsync(dtv + n, s->S.dt, sizeof(double), cudaMemcpyDeviceToDevice, q));
        launch_adj_record(s->M, s->S, s->P, rp + (size_t)n * nc, pf + (size_t)n * 5 * nc, q);
    }
    rc = read_error(s);
    if (rc) return rc;
    std::vector<double> dth(K);
    CU(cudaMemcpyAsync(dth.data(), dtv, K * sizeof(double), cudaMemcpyDeviceToHost, q));
    CU(cudaStreamSynchronize(q));
    // 2. frozen forward at theta: checkpoints and the functional
    for (int n = 0; n < K; ++n)
        launch_adj_forward(s->M, s->P, ap, ck + (size_t)n * 5 * nc, rp + (size_t)n * nc, pf + (size_t)n * 5 * nc, dth[n],
                           theta, step_o2(n), F, jf, sums + n, ck + (size_t)(n + 1) * 5 * nc, q);
    // 3. reverse sweep
    CU(cudaMemsetAsync(lam1, 0, 5 * nc * sizeof(double), q));
    double* next = lam1;
    double* cur = lam0;
    for (int n = K - 1; n >= 0; --n) {
        launch_adj_reverse(s->M, s->P, ap, ck + (size_t)n * 5 * nc, rp + (size_t)n * nc, dth[n], theta, step_o2(n), next,
                           cur, wbar, thbar, sums + K + 3 * (size_t)n, q);
        std::swap(next, cur);
    }
    CU(cudaGetLastError());
    std::vector<double> h(4 * (size_t)K);
    CU(cudaMemcpyAsync(h.data(), sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, q));
    CU(cudaStreamSynchronize(q));
    out[0] = 0.0;
    out[1] = out[2] = out[3] = 0.0;
    for (int n = 0; n < K; ++n) {
        out[0] += h[n];
        for (int k = 0; k < 3; ++k) out[1 + k] += h[K + 3 * (size_t)n + k];
    }
    return UGKWP_OK;
}

}  // extern "C"

// ------------------------------------------------------ launch configuration
extern "C" {

int ugkwp_get_launch_cfg(const ugkwp_sim* s, ugkwp_launch_cfg* out) {
    if (!s || !out) return fail(UGKWP_E_ARG, "NULL argument");
    out->particle_blocks = s->lc.particle_blocks;
    out->wave_blocks = s->lc.wave_blocks;
    out->track_threads = s->lc.track.threads;
    out->smem_carveout = s->lc.carveout;
    return UGKWP_OK;
}

int ugkwp_set_launch_cfg(ugkwp_sim* s, const ugkwp_launch_cfg* cfg) {
    if (!s || !cfg) return fail(UGKWP_E_ARG, "NULL argument");
    if (cfg->particle_blocks <= 0 || cfg->wave_blocks <= 0 || cfg->particle_blocks > (1 << 20) ||
        cfg->wave_blocks > (1 << 20))
        return fail(UGKWP_E_ARG, "grid sizes must be in [1, 2^20]");
    if (cfg->track_threads != 128 && cfg->track_threads != 256)
        return fail(UGKWP_E_ARG, "track_threads must be 128 or 256");
    if (cfg->smem_carveout < -1 || cfg->smem_carveout > 100)
        return fail(UGKWP_E_ARG, "smem_carveout must be -1 or in [0, 100]");
    LaunchCfg lc{cfg->particle_blocks, cfg->wave_blocks, TrackShape{cfg->track_threads}, cfg->smem_carveout};
    if (lc.particle_blocks != s->lc.particle_blocks || lc.wave_blocks != s->lc.wave_blocks ||
        lc.track.threads != s->lc.track.threads || lc.carveout != s->lc.carveout) {
        CU(configure_kernels(s->P, lc));
        s->lc = lc;
        s->drop_graphs();
    }
    return UGKWP_OK;
}

}  // extern "C"

namespace {

ugkwp_launch_cfg to_public(const LaunchCfg& c) {
    return ugkwp_launch_cfg{c.particle_blocks, c.wave_blocks, c.track.threads, c.carveout};
}

// The autotuner's search, in two stages: (1) tracking block shape x carveout
// at 1024 resident tracking threads per SM and one wave block per SM; (2) for the
// fastest of those, resident tracking threads per SM (512, 1024, 2048) x wave
// blocks per SM (1, 2 at order 2).  trial(c, ms) sets c, steps and returns the
// time; the fastest configuration is returned in best.
template <class Trial> int tune_search(int order, Trial&& trial, LaunchCfg& best) {
    const int sms = sm_count();
    const TrackShape shapes[] = {{128}, {256}};
    float best_ms = 0.0f;
    bool have = false;
    auto consider = [&](const LaunchCfg& c) {
        float ms = 0.0f;
        int rc = trial(c, ms);
        if (rc) return rc;
        if (!have || ms < best_ms) { best_ms = ms; best = c; have = true; }
        return (int)UGKWP_OK;
    };
    for (const TrackShape& sh : shapes)
        for (int carve : {-1, 58}) {
            int rc = consider(LaunchCfg{1024 / sh.threads * sms, sms, sh, carve});
            if (rc) return rc;
        }
    const LaunchCfg stage1 = best;
    for (int threads_per_sm : {512, 1024, 2048})
        for (int wb : {1, 2}) {
            if (order != 2 && wb != 1) continue;
            if (threads_per_sm == 1024 && wb == 1) continue;  // measured in the first stage
            int rc = consider(LaunchCfg{threads_per_sm / stage1.track.threads * sms, wb * sms, stage1.track,
                                        stage1.carveout});
            if (rc) return rc;
        }
    return UGKWP_OK;
}

// Device time of `steps` steps enqueued by `run` on stream q.
template <class F> int time_steps(cudaStream_t q, F&& run, float& ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    CU(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(UGKWP_E_CUDA, "cudaEventCreate");
    }
    int rc = UGKWP_OK;
    if (cudaEventRecord(a, q) != cudaSuccess) rc = fail(UGKWP_E_CUDA, "cudaEventRecord");
    if (rc == UGKWP_OK) rc = run();
    if (rc == UGKWP_OK && cudaEventRecord(b, q) != cudaSuccess) rc = fail(UGKWP_E_CUDA, "cudaEventRecord");
    if (rc == UGKWP_OK && cudaEventSynchronize(b) != cudaSuccess) rc = fail(UGKWP_E_CUDA, "cudaEventSynchronize");
    if (rc == UGKWP_OK && cudaEventElapsedTime(&ms, a, b) != cudaSuccess) rc = fail(UGKWP_E_CUDA, "cudaEventElapsedTime");
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}

}  // namespace

extern "C" {

int ugkwp_autotune(ugkwp_sim* s, int32_t steps_per_trial, ugkwp_launch_cfg* best) {
    if (!s) return fail(UGKWP_E_ARG, "NULL simulation");
    if (steps_per_trial < 2 || (steps_per_trial & 1)) return fail(UGKWP_E_ARG, "steps_per_trial must be even and >= 2");
    if (s->timing) return fail(UGKWP_E_STATE, "per-kernel timing is enabled");
    LaunchCfg best_lc = s->lc;
    int rc = tune_search(s->P.order, [&](const LaunchCfg& c, float& ms) {
        ugkwp_launch_cfg u = to_public(c);
        int r = ugkwp_set_launch_cfg(s, &u);
        if (r) return r;
        r = ugkwp_step(s, 2, nullptr);
        if (r) return r;
        r = time_steps(s->stream, [&] { return ugkwp_step(s, steps_per_trial, nullptr); }, ms);
        if (r) return r;
        return read_error(s);
    }, best_lc);
    if (rc) return rc;
    ugkwp_launch_cfg u = to_public(best_lc);
    rc = ugkwp_set_launch_cfg(s, &u);
    if (rc) return rc;
    if (best) *best = u;
    return UGKWP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
// Members of a batch that share precision, order, K > 0 and sampling form
// fused chunks of up to BATCH_CHUNK members: each kernel of the step is one
// launch for the whole chunk, on the chunk's own streams.
struct FusedChunk {
    std::vector<int> idx;  // members (indices into the batch)
    int precision = 0, order = 1, sampling = 0;
    bool ke = false;
    cudaStream_t lane = nullptr, wave = nullptr, aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, sampled = nullptr, tracked = nullptr, gp_ready = nullptr,
                done = nullptr, waved = nullptr;
    ~FusedChunk() {
        for (cudaEvent_t e : {fork, join, sampled, tracked, gp_ready, done, waved})
            if (e) cudaEventDestroy(e);
        for (cudaStream_t q : {lane, wave, aux})
            if (q) cudaStreamDestroy(q);
    }
};

struct ugkwp_batch {
    std::vector<ugkwp_sim*> sims;
    cudaStream_t stream = nullptr;
    std::vector<cudaStream_t> lanes;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    std::vector<std::unique_ptr<FusedChunk>> chunks;
    // two-step graphs keyed by every member's buffer A (ping-pong parities)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::vector<void*> key[2];
    std::vector<std::vector<int64_t>> launches[2];  // per member, per kernel class
    void drop_graphs() {
        for (int k = 0; k < 2; ++k) {
            if (graph[k]) cudaGraphExecDestroy(graph[k]);
            graph[k] = nullptr;
            key[k].clear();
            launches[k].clear();
        }
    }
    ~ugkwp_batch() {
        if (stream) cudaStreamSynchronize(stream);
        drop_graphs();
        for (auto e : join) if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (auto l : lanes) if (l) cudaStreamDestroy(l);
    }
};

namespace {

// A batch graph holds every member's structures as they were at capture: it
// is valid while each member's step parity and structure generation match.
std::vector<void*> batch_key(const ugkwp_batch* b) {
    std::vector<void*> k;
    k.reserve(2 * b->sims.size());
    for (auto* s : b->sims) {
        k.push_back(s->S.nleft);
        k.push_back(reinterpret_cast<void*>(static_cast<uintptr_t>(s->gen)));
    }
    return k;
}

// Proportional split of `total` blocks over members of work w[i] (at least one
// block each, at most need[i]).
std::vector<int> split_blocks(int total, const std::vector<long long>& w, const std::vector<int>& need) {
    long long W = 0;
    for (long long v : w) W += v;
    std::vector<int> out(w.size(), 1);
    for (size_t i = 0; i < w.size(); ++i) {
        long long v = W > 0 ? (long long)total * w[i] / W : 1;
        if (v < 1) v = 1;
        if (v > need[i]) v = need[i];
        out[i] = (int)v;
    }
    return out;
}

// One step of a fused chunk, enqueued like enqueue_step for a single
// simulation: the same kernels in the same stream order, each one launch
// for all members of the chunk.
int enqueue_chunk_step(FusedChunk& ch, const std::vector<ugkwp_sim*>& sims) {
    BatchChunk c;
    std::memset(&c, 0, sizeof(c));
    c.n = (int32_t)ch.idx.size();
    const LaunchCfg lc = sims[ch.idx[0]]->lc;
    const int sms = sm_count();
    std::vector<long long> w6(c.n), wf(c.n);
    std::vector<int> need_grad(c.n), need_o2(c.n), need_o1(c.n);
    for (int i = 0; i < c.n; ++i) {
        ugkwp_sim* s = sims[ch.idx[i]];
        c.mem[i] = BatchMember{s->M, s->S, s->P, s->A, s->B, s->Mv};
        w6[i] = 6LL * s->M.nc;
        wf[i] = s->M.nf;
        need_grad[i] = (int)((6LL * s->M.nc + gradient_threads() - 1) / gradient_threads());
        need_o2[i] = (s->M.nf + wave_threads() - 1) / wave_threads();
        need_o1[i] = (s->M.nf + 255) / 256;
    }
    const std::vector<int> b_grad = split_blocks(4 * sms, w6, need_grad);
    const std::vector<int> b_o2 = split_blocks(lc.wave_blocks, wf, need_o2);
    const std::vector<int> b_o1 = split_blocks(lc.wave_blocks, wf, need_o1);
    for (int k = 0; k < BCL_N; ++k) c.off[k][0] = 0;
    for (int i = 0; i < c.n; ++i) {
        const int nc = c.mem[i].m.nc;
        const int per[BCL_N] = {blocks_reset(nc), blocks_cells(nc), scan_blocks(nc), b_grad[i], blocks_gp_coef(nc),
                                b_o2[i], b_o1[i]};
        for (int k = 0; k < BCL_N; ++k) c.off[k][i + 1] = c.off[k][i] + per[k];
    }
    auto blocks = [&](int k) { return c.off[k][c.n]; };
    cudaStream_t q = ch.lane;
    launch_reset_batch(c, blocks(BCL_RESET), q);
    launch_cell_prep_batch(c, blocks(BCL_CELLS), q);
    launch_sample_count_batch(c, blocks(BCL_SCAN), q);
    CU(cudaEventRecord(ch.fork, q));
    CU(cudaStreamWaitEvent(ch.wave, ch.fork, 0));
    const bool gp = ch.sampling == UGKWP_SAMPLE_GP1;
    if (ch.order == 2) {
        launch_gradients_batch(c, blocks(BCL_GRAD), ch.wave);
        if (gp) launch_gp_coef_batch(c, blocks(BCL_GPC), ch.wave);
    }
    if (gp) CU(cudaEventRecord(ch.gp_ready, ch.wave));
    if (ch.order == 2) launch_face_flux_o2_batch(c, blocks(BCL_FLUX_O2), ch.wave);
    else launch_face_flux_batch(c, blocks(BCL_FLUX), ch.wave);
    CU(cudaEventRecord(ch.join, ch.wave));
    launch_wave_update_batch(c, blocks(BCL_CELLS), ch.wave);
    CU(cudaEventRecord(ch.waved, ch.wave));
    launch_scan_batch(c, blocks(BCL_SCAN), q);
    if (gp) CU(cudaStreamWaitEvent(q, ch.gp_ready, 0));
    if (ch.sampling == UGKWP_SAMPLE_ENERGY_MATCHED) launch_sample_scale_batch(c, blocks(BCL_CELLS), ch.precision, q);
    launch_sample_write_batch(c, lc.particle_blocks, ch.precision, q);
    const int first_half = (lc.particle_blocks + 1) / 2;
    CU(cudaEventRecord(ch.sampled, q));
    launch_track_batch(c, ch.precision, ch.ke, lc.track, first_half, q);
    CU(cudaStreamWaitEvent(ch.aux, ch.sampled, 0));
    CU(cudaStreamWaitEvent(ch.aux, ch.join, 0));
    if (lc.particle_blocks > first_half)
        launch_track_batch(c, ch.precision, ch.ke, lc.track, lc.particle_blocks - first_half, ch.aux);
    CU(cudaEventRecord(ch.tracked, ch.aux));
    CU(cudaStreamWaitEvent(q, ch.tracked, 0));
    launch_movers_batch(c, lc.particle_blocks, ch.precision, q);
    CU(cudaStreamWaitEvent(q, ch.waved, 0));
    launch_cell_update_batch(c, blocks(BCL_CELLS), q);
    for (int i = 0; i < c.n; ++i) {
        ugkwp_sim* s = sims[ch.idx[i]];
        std::swap(s->A, s->B);
        std::swap(s->S.nleft, s->S.nleft_next);
        std::swap(s->S.smass, s->S.smass_next);
    }
    return UGKWP_OK;
}

bool batch_graphs_allowed(const ugkwp_batch* b) {
    for (auto* s : b->sims)
        if (s->timing || !s->graphs_ok) return false;
    return true;
}

// Enqueue `n` (1 or 2) steps of every member on the batch's lanes, forked from
// and joined back into the batch stream: as fused chunks, or (while a member
// records per-kernel times) as each member's own kernels.
int batch_enqueue(ugkwp_batch* b, int n) {
    CU(cudaEventRecord(b->fork, b->stream));
    bool timing = false;
    for (auto* s : b->sims) timing = timing || s->timing;
    if (!timing && !b->chunks.empty()) {
        for (auto& ch : b->chunks) {
            CU(cudaStreamWaitEvent(ch->lane, b->fork, 0));
            for (int k = 0; k < n; ++k) {
                int rc = enqueue_chunk_step(*ch, b->sims);
                if (rc) return rc;
            }
            CU(cudaEventRecord(ch->done, ch->lane));
            CU(cudaStreamWaitEvent(b->stream, ch->done, 0));
        }
        return UGKWP_OK;
    }
    const size_t L = b->lanes.size();
    for (size_t i = 0; i < b->sims.size(); ++i) {
        ugkwp_sim* s = b->sims[i];
        cudaStream_t lane = b->lanes[i % L];
        CU(cudaStreamWaitEvent(lane, b->fork, 0));
        cudaStream_t own = s->stream;
        s->stream = lane;
        int rc = UGKWP_OK;
        for (int k = 0; k < n && rc == UGKWP_OK; ++k) rc = enqueue_step(s);
        s->stream = own;
        if (rc) return rc;
        CU(cudaEventRecord(b->join[i], lane));
        CU(cudaStreamWaitEvent(b->stream, b->join[i], 0));
    }
    return UGKWP_OK;
}

int batch_step_pair(ugkwp_batch* b, bool& used) {
    used = false;
    if (!batch_graphs_allowed(b)) return UGKWP_OK;
    const std::vector<void*> k = batch_key(b);
    int slot = b->key[0] == k ? 0 : b->key[1] == k ? 1 : -1;
    if (slot < 0) {
        slot = b->graph[0] ? 1 : 0;
        if (b->graph[slot]) { cudaGraphExecDestroy(b->graph[slot]); b->graph[slot] = nullptr; }
        std::vector<std::vector<int64_t>> saved(b->sims.size());
        for (size_t i = 0; i < b->sims.size(); ++i)
            saved[i].assign(b->sims[i]->launches, b->sims[i]->launches + UGKWP_N_KERNELS);
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return UGKWP_OK;
        }
        int rc = batch_enqueue(b, 2);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        b->launches[slot].assign(b->sims.size(), std::vector<int64_t>(UGKWP_N_KERNELS, 0));
        for (size_t i = 0; i < b->sims.size(); ++i)
            for (int c = 0; c < UGKWP_N_KERNELS; ++c) {
                b->launches[slot][i][c] = b->sims[i]->launches[c] - saved[i][c];
                b->sims[i]->launches[c] = saved[i][c];
            }
        if (rc != UGKWP_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc;
        }
        e = cudaGraphInstantiate(&b->graph[slot], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->graph[slot] = nullptr;
            return UGKWP_OK;
        }
        b->key[slot] = k;
    }
    CU(cudaGraphLaunch(b->graph[slot], b->stream));
    for (size_t i = 0; i < b->sims.size(); ++i)
        for (int c = 0; c < UGKWP_N_KERNELS; ++c) b->sims[i]->launches[c] += b->launches[slot][i][c];
    used = true;
    return UGKWP_OK;
}

}  // namespace

extern "C" {

int ugkwp_batch_create(ugkwp_sim* const* sims, int32_t n_sims, void* cuda_stream, ugkwp_batch** out) {
    if (!out) return fail(UGKWP_E_ARG, "NULL argument");
    *out = nullptr;
    if (!sims || n_sims <= 0) return fail(UGKWP_E_ARG, "a batch needs at least one simulation");
    std::vector<ugkwp_sim*> v(sims, sims + n_sims);
    for (auto* s : v)
        if (!s) return fail(UGKWP_E_ARG, "NULL simulation in the batch");
    std::vector<ugkwp_sim*> sorted = v;
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
        return fail(UGKWP_E_ARG, "a simulation appears twice in the batch");
    ugkwp_batch* b = new ugkwp_batch;
    b->sims = v;
    b->stream = (cudaStream_t)cuda_stream;
    const int n_lanes = std::min(n_sims, 32);
    cudaError_t ce = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < n_lanes && ce == cudaSuccess; ++i) {
        cudaStream_t l = nullptr;
        ce = cudaStreamCreateWithFlags(&l, cudaStreamNonBlocking);
        b->lanes.push_back(l);
    }
    b->join.assign(v.size(), nullptr);
    for (size_t i = 0; i < v.size() && ce == cudaSuccess; ++i) ce = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    // fused chunks: members grouped by precision, order, K > 0 and sampling,
    // in batch order, at most BATCH_CHUNK per chunk
    for (size_t i = 0; i < v.size() && ce == cudaSuccess; ++i) {
        const DevParams& P = v[i]->P;
        FusedChunk* into = nullptr;
        for (auto& ch : b->chunks)
            if (ch->precision == P.precision && ch->order == P.order && ch->ke == (P.K > 0) &&
                ch->sampling == P.sampling && (int)ch->idx.size() < BATCH_CHUNK)
                into = ch.get();
        if (!into) {
            b->chunks.emplace_back(new FusedChunk);
            into = b->chunks.back().get();
            into->precision = P.precision;
            into->order = P.order;
            into->ke = P.K > 0;
            into->sampling = P.sampling;
            for (cudaStream_t* q : {&into->lane, &into->wave, &into->aux})
                if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(q, cudaStreamNonBlocking);
            // the fork is a timing event, as a single simulation's is
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&into->fork, cudaEventDefault);
            for (cudaEvent_t* e : {&into->join, &into->sampled, &into->tracked, &into->gp_ready, &into->done, &into->waved})
                if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
        }
        into->idx.push_back((int)i);
    }
    if (ce != cudaSuccess) {
        delete b;
        return cuda_fail(ce, "ugkwp_batch_create");
    }
    *out = b;
    return UGKWP_OK;
}

int ugkwp_batch_step(ugkwp_batch* b, int32_t n_steps) {
    if (!b || n_steps < 0) return fail(UGKWP_E_ARG, "invalid argument");
    for (auto* s : b->sims)
        if (s->step + n_steps >= ((int64_t)1 << 24) - 2) return fail(UGKWP_E_STATE, "step counter exhausted (2^24 steps)");
    for (int32_t k = 0; k < n_steps;) {
        if (n_steps - k >= 2) {
            bool used = false;
            int rc = batch_step_pair(b, used);
            if (rc) return rc;
            if (used) {
                for (auto* s : b->sims) s->step += 2;
                k += 2;
                continue;
            }
        }
        int rc = batch_enqueue(b, 1);
        if (rc) return rc;
        for (auto* s : b->sims) s->step += 1;
        k += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return UGKWP_OK;
}

int ugkwp_batch_sync(ugkwp_batch* b) {
    if (!b) return fail(UGKWP_E_ARG, "NULL batch");
    CU(cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < b->sims.size(); ++i) {
        int rc = read_error(b->sims[i]);
        if (rc) return fail(rc, "batch member " + std::to_string(i) + ": " + g_err);
    }
    return UGKWP_OK;
}

int ugkwp_batch_autotune(ugkwp_batch* b, int32_t steps_per_trial, ugkwp_launch_cfg* best) {
    if (!b) return fail(UGKWP_E_ARG, "NULL batch");
    if (steps_per_trial < 2 || (steps_per_trial & 1)) return fail(UGKWP_E_ARG, "steps_per_trial must be even and >= 2");
    int order = 1;
    for (auto* s : b->sims) {
        if (s->timing) return fail(UGKWP_E_STATE, "per-kernel timing is enabled on a member");
        order = std::max(order, (int)s->P.order);
    }
    LaunchCfg best_lc = b->sims.empty() ? LaunchCfg{1, 1, {128}, -1} : b->sims[0]->lc;
    int rc0 = tune_search(order, [&](const LaunchCfg& c, float& ms) {
        ugkwp_launch_cfg u = to_public(c);
        for (auto* s : b->sims) {
            int r = ugkwp_set_launch_cfg(s, &u);
            if (r) return r;
        }
        b->drop_graphs();
        int r = ugkwp_batch_step(b, 2);
        if (r) return r;
        r = time_steps(b->stream, [&] { return ugkwp_batch_step(b, steps_per_trial); }, ms);
        if (r) return r;
        return ugkwp_batch_sync(b);
    }, best_lc);
    if (rc0) return rc0;
    ugkwp_launch_cfg u = to_public(best_lc);
    for (auto* s : b->sims) {
        int rc = ugkwp_set_launch_cfg(s, &u);
        if (rc) return rc;
    }
    b->drop_graphs();
    if (best) *best = u;
    return UGKWP_OK;
}

int ugkwp_batch_free(ugkwp_batch* b) {
    delete b;
    return UGKWP_OK;
}

}  // extern "C"
