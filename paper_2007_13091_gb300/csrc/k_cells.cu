// Per-cell kernels of the UGKWP step: primitives, relaxation time and the
// time-step reduction (a1, a2), hydro-particle counts (a5), the exclusive scan
// that places each cell's samples after the survivors (a11), and the
// conservative update (a10).  Compiled with --fmad=false: tau, dt, N_sam and m_sam decide integer
// outcomes of the particle path and must be reproducible bit for bit.
#include <cfloat>

#include "dmath.cuh"
#include "ugkwp_internal.hpp"

namespace ugkwp {

namespace {

__device__ __forceinline__ void set_err(const DevState& s, int32_t bits) {
    atomicOr(reinterpret_cast<unsigned long long*>(&s.cnt64[CNT_ERR]), (unsigned long long)bits);
}

// Inclusive scan of two ints per thread (count, N_sam) over one block.
__device__ __forceinline__ int2 block_scan_incl2(int2 v, int2* sh_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int ox = __shfl_up_sync(0xffffffffu, v.x, d);
        const int oy = __shfl_up_sync(0xffffffffu, v.y, d);
        if (lane >= d) { v.x += ox; v.y += oy; }
    }
    if (lane == 31) sh_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int2 w = (lane < (int)(blockDim.x >> 5)) ? sh_warp[lane] : make_int2(0, 0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int ox = __shfl_up_sync(0xffffffffu, w.x, d);
            const int oy = __shfl_up_sync(0xffffffffu, w.y, d);
            if (lane >= d) { w.x += ox; w.y += oy; }
        }
        sh_warp[lane] = w;
    }
    __syncthreads();
    if (warp > 0) { v.x += sh_warp[warp - 1].x; v.y += sh_warp[warp - 1].y; }
    return v;
}

__device__ __forceinline__ void reset_body(const DevMesh& m, const DevState& s, Blk bk) {
    const int nc = m.nc;
    const long long stride = (long long)bk.n * blockDim.x;
    for (long long i = (long long)bk.id * blockDim.x + threadIdx.x; i < 5LL * nc; i += stride) {
        s.pflux[i] = 0;
        if (i < nc) {
            s.nleft_next[i] = 0;
            s.smass_next[i] = 0;
        }
    }
    if (bk.id == 0 && threadIdx.x == 0) {
        s.cnt64[CNT_SAMPLED] = 0;
        s.cnt64[CNT_COLLIDED] = 0;
        s.cnt64[CNT_EXITED] = 0;
        s.cnt64[CNT_LOST] = 0;
        s.cnt64[CNT_CROSSINGS] = 0;
        s.cnt64[CNT_WALL] = 0;
        s.cnt64[CNT_RESV] = 0;
        s.cnt64[CNT_TRACKED] = 0;
        s.cnt64[CNT_DT_BITS] = 0x7ff0000000000000LL;  // +inf
        s.cnt64[CNT_TILE] = 0;
        s.cnt64[CNT_OVF] = 0;
        s.cnt64[CNT_SURV] = 0;
    }
}
__global__ void k_reset(DevMesh m, DevState s) {
    reset_body(m, s, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// a1 + a2: primitives, tau = mu_ref/p (T/T_ref)^omega, rho^p from the survivors'
// fixed-point mass, rho^h = rho - rho^p, and min_i |Omega_i| / sum_d Lambda_i^d.
__device__ __forceinline__ void cell_prep_body(const DevMesh& m, const DevState& s, const DevParams& p, Blk bk) {
    const int nc = m.nc;
    const int i = bk.id * blockDim.x + threadIdx.x;
    double r = __longlong_as_double(0x7ff0000000000000LL);
    if (i < nc) {
        const double rho = s.W[i];
        const double Ux = s.W[nc + i] / rho, Uy = s.W[2 * nc + i] / rho, Uz = s.W[3 * nc + i] / rho;
        const double U2 = (Ux * Ux + Uy * Uy) + Uz * Uz;
        const double pr = (s.W[4 * nc + i] - 0.5 * (rho * U2)) / (1.5 + 0.5 * (double)p.K);
        const double T = pr / (rho * p.R);
        double tau = 1.0;
        if (!(rho > 0.0) || !(pr > 0.0) || !isfinite(pr)) {
            set_err(s, ERRB_NONFINITE);
        } else {
            tau = (p.mu_ref / pr) * dm::d_exp(p.omega * dm::d_log(T / p.T_ref));
            const double c = 3.0 * sqrt(p.R * T);
            const double lam = ((fabs(Ux) + c) * m.dS[i] + (fabs(Uy) + c) * m.dS[nc + i]) + (fabs(Uz) + c) * m.dS[2 * nc + i];
            r = m.vol[i] / lam;
        }
        if (p.gks == 2) s.dtc[i] = p.CFL * r;
        const double rhop = ((double)s.smass[i] * p.qscale[0]) / m.vol[i];
        s.prim[i] = rho;
        s.prim[nc + i] = Ux;
        s.prim[2 * nc + i] = Uy;
        s.prim[3 * nc + i] = Uz;
        s.prim[4 * nc + i] = T;
        s.tau[i] = tau;
        s.tauf[i] = (float)tau;
        if (p.precision == UGKWP_MIXED)
            s.usig[i] = make_float4((float)Ux, (float)Uy, (float)Uz, (float)sqrt(p.R * T));
        s.rhop[i] = rhop;
        s.rhoh[i] = rho - rhop;
    }
    // block minimum, then one atomic on the ordered bit pattern (r > 0)
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) r = fmin(r, __shfl_xor_sync(0xffffffffu, r, d));
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, d));
        if (threadIdx.x == 0 && v < __longlong_as_double(0x7ff0000000000000LL) && v > 0.0)
            atomicMin(reinterpret_cast<unsigned long long*>(&s.cnt64[CNT_DT_BITS]),
                      (unsigned long long)__double_as_longlong(v));
    }
}
__global__ void k_cell_prep(DevMesh m, DevState s, DevParams p) {
    cell_prep_body(m, s, p, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// a5 counts: rho^hp = e^{-dt/tau} rho^h, m_ref = (rho^p + rho^hp)|Omega|/N_ref,
// N_sam = 2 ceil(rho^hp |Omega| / (2 m_ref)), N_sam >= N_min - N_left,
// m_sam = rho^hp |Omega| / N_sam (Sec. 2.4 (b)).  Also the survivor bucket
// the cell gets in the buffer this step's survivors are written to (a11:
// sized from the particles that start the step in the cell), and the
// per-block sums of the bucket sizes and of N_sam.
__device__ __forceinline__ void sample_count_body(const DevMesh& m, const DevState& s, const DevParams& p, Blk bk) {
    __shared__ int2 shw[32];
    const int nc = m.nc;
    const int i = bk.id * blockDim.x + threadIdx.x;
    const double dt = p.CFL * __longlong_as_double(s.cnt64[CNT_DT_BITS]);
    if (p.gks) {  // GKS step: the time step only, nothing is sampled
        if (i == 0) s.dt[0] = dt;
        return;
    }
    int wcap = 0, nsam = 0;
    if (i < nc) {
        const double vol = m.vol[i];
        const double ex = dm::d_exp(-(dt / s.tau[i]));
        const double rh = s.rhoh[i] > 0.0 ? s.rhoh[i] : 0.0;
        const double rhp = ex * rh;
        const double Mhp = rhp * vol;
        long long ns = 0;
        double ms = 0.0;
        if (Mhp > (s.prim[i] * vol) * 0x1p-30) {
            const double mref = ((s.rhop[i] + rhp) * vol) / (double)p.N_ref;
            ns = 2 * (long long)ceil(Mhp / (2.0 * mref));
            const long long need = (long long)p.N_min - (long long)s.nleft[i];
            if (need > ns) ns = need + (need & 1);
            if (ns > 65534) {
                set_err(s, ERRB_SAMPLE_LIMIT);
                ns = 0;
            } else {
                ms = Mhp / (double)ns;
            }
        }
        s.nsam[i] = (int)ns;
        s.msam[i] = ms;
        nsam = (int)ns;
        const int count = s.nleft[i] + nsam;
        s.cnt[i] = count;
        wcap = bucket_slots(count);
        s.wcap[i] = wcap;
    }
    const int2 incl = block_scan_incl2(make_int2(wcap, nsam), shw);
    if (threadIdx.x == blockDim.x - 1) s.bsum[bk.id] = incl;
    if (i == 0) s.dt[0] = dt;
}
__global__ void k_sample_count(DevMesh m, DevState s, DevParams p) {
    sample_count_body(m, s, p, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// Exclusive scan of the block sums (one block): the slots of the survivor
// buckets of the buffer written this step and the sampled particles (they
// follow the N_A slots of the current buffer), and the capacity checks.
__device__ __forceinline__ void scan_bsum_body(const DevState& s, const DevParams& p, int nb) {
    __shared__ int2 shw[32];
    __shared__ long long carry_sh[2];
    if (threadIdx.x == 0) { carry_sh[0] = 0; carry_sh[1] = 0; }
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        const int j = base + threadIdx.x;
        const int2 v = j < nb ? s.bsum[j] : make_int2(0, 0);
        const int2 incl = block_scan_incl2(v, shw);
        const long long c0 = carry_sh[0], c1 = carry_sh[1];
        if (j < nb) s.bsum[j] = make_int2((int)(c0 + incl.x - v.x), (int)(c1 + incl.y - v.y));
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) { carry_sh[0] = c0 + incl.x; carry_sh[1] = c1 + incl.y; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long total = s.cnt64[CNT_N_A] + carry_sh[1];
        s.cnt64[CNT_N_B] = total;
        s.cnt64[CNT_NSAM] = carry_sh[1];
        s.cnt64[CNT_SAMPLED] = carry_sh[1];
        s.cnt64[CNT_WTOT] = carry_sh[0];
        if (total > p.capacity || carry_sh[0] > p.capacity) {
            set_err(s, ERRB_CAPACITY);
            s.cnt64[CNT_N_B] = 0;
            s.cnt64[CNT_NSAM] = 0;
        }
    }
}
__global__ void k_scan_bsum(DevState s, DevParams p, int nb) {
    scan_bsum_body(s, p, nb);
}

__device__ __forceinline__ void scan_apply_body(const DevMesh& m, const DevState& s, Blk bk) {
    __shared__ int2 shw[32];
    const int i = bk.id * blockDim.x + threadIdx.x;
    const int2 v = i < m.nc ? make_int2(s.wcap[i], s.nsam[i]) : make_int2(0, 0);
    const int2 incl = block_scan_incl2(v, shw);
    if (i < m.nc) {
        s.soff[i] = s.bsum[bk.id].y + incl.y - v.y;
        s.woff[i] = s.bsum[bk.id].x + incl.x - v.x;
    }
}
__global__ void k_scan_apply(DevMesh m, DevState s) {
    scan_apply_body(m, s, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// a10: W^{n+1} = W^n - 1/|Omega| sum_k (+-F_k |S_k|) + F^{fr,p}/|Omega|, faces
// gathered in local order 0..3 (Eq. update_macro_variables).
__device__ __forceinline__ void cell_update_body(const DevMesh& m, const DevState& s, const DevParams& p, int32_t* wcell, Blk bk) {
    const int nc = m.nc, nf = m.nf;
    const int i = bk.id * blockDim.x + threadIdx.x;
    if (p.gks) {
        // GKS step (no particles): W -= sum_k (+-F_k |S_k|) / |Omega|; with local
        // steps F_k holds the flux rate and the cell advances by its own dt
        if (i == 0 && p.gks == 1) s.t[0] = s.t[0] + s.dt[0];
        if (i >= nc) return;
        const int own = m.cfs[i];
        const double vol = m.vol[i];
        for (int q = 0; q < 5; ++q) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) {
                const int f = m.cf[k * nc + i];
                const double v = s.F[(size_t)q * nf + f] * m.f_area[f];
                acc = acc + (((own >> k) & 1) ? v : -v);
            }
            double& w = s.W[(size_t)q * nc + i];
            w = p.gks == 2 ? w - (s.dtc[i] * acc) / vol : w - acc / vol;
        }
        return;
    }
    if (i == 0) {
        s.t[0] = s.t[0] + s.dt[0];
        if (p.averaging) s.tsum[0] += s.dt[0];
        s.cnt64[CNT_STEP] += 1;
        // the survivor buckets and the overflow slots become the current buffer
        const long long ovf = s.cnt64[CNT_OVF];
        const long long room = p.capacity - s.cnt64[CNT_WTOT];
        s.cnt64[CNT_N_A] = s.cnt64[CNT_WTOT] + (ovf < room ? ovf : room);
    }
    if (i >= nc) return;
    // a11: the bucket slots no survivor took are holes
    if (!(s.cnt64[CNT_ERR] & ERRB_CAPACITY)) {
        const int cap = s.wcap[i], fill = s.nleft_next[i];
        if ((long long)s.woff[i] + cap <= p.capacity)
            for (int k = fill < cap ? fill : cap; k < cap; ++k) wcell[(size_t)s.woff[i] + k] = -1;
    }
    // the particle part, added to W - sum_k (+-F_k |S_k|) / |Omega| that
    // k_wave_update left in W: (W - acc/|Omega|) + F^{fr,p}/|Omega|
    const double ivol = m.ivol[i];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double fp = (double)s.pflux[(size_t)q * nc + i] * p.qscale[q];
        double& w = s.W[(size_t)q * nc + i];
        w = w + fp * ivol;
        if (p.averaging) s.wsum[(size_t)q * nc + i] += s.dt[0] * w;
    }
}

// a10, the wave part of a step with particles: W <- W - sum_k (+-F_k |S_k|)
// |Omega|^-1, faces gathered in local order 0..3.  It runs as soon as the
// wave flux is done, beside the tracking (no particle kernel reads W);
// k_cell_update adds the particle part once the movers' flux is summed.
__device__ __forceinline__ void wave_update_body(const DevMesh& m, const DevState& s, Blk bk) {
    const int nc = m.nc, nf = m.nf;
    const int i = bk.id * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    int f[4];
    const int own = m.cfs[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) f[k] = m.cf[k * nc + i];
    // 1/|Omega| once per cell (the factor of the update) instead of ten
    // binary64 divisions
    const double ivol = m.ivol[i];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double v = s.F[(size_t)q * nf + f[k]] * m.f_area[f[k]];
            acc = acc + (((own >> k) & 1) ? v : -v);
        }
        double& w = s.W[(size_t)q * nc + i];
        w = w - acc * ivol;
    }
}
__global__ void k_wave_update(DevMesh m, DevState s) {
    wave_update_body(m, s, Blk{(int)blockIdx.x, (int)gridDim.x});
}
__global__ void k_cell_update(DevMesh m, DevState s, DevParams p, int32_t* wcell) {
    cell_update_body(m, s, p, wcell, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// ---- fused batches: member i of the chunk runs on the blocks
// off[cls][i] .. off[cls][i + 1] - 1, the grid its own launch would have.
__device__ __forceinline__ int member_of(const int32_t* off, int n) {
    int lo = 0, hi = n;  // off[lo] <= blockIdx.x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ Blk member_blk(const int32_t* off, int i) {
    return Blk{(int)blockIdx.x - off[i], off[i + 1] - off[i]};
}

__global__ void k_reset_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_RESET], c.n);
    reset_body(c.mem[i].m, c.mem[i].s, member_blk(c.off[BCL_RESET], i));
}
__global__ void k_cell_prep_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_CELLS], c.n);
    cell_prep_body(c.mem[i].m, c.mem[i].s, c.mem[i].p, member_blk(c.off[BCL_CELLS], i));
}
__global__ void k_sample_count_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_SCAN], c.n);
    sample_count_body(c.mem[i].m, c.mem[i].s, c.mem[i].p, member_blk(c.off[BCL_SCAN], i));
}
// one block per member
__global__ void k_scan_bsum_b(const __grid_constant__ BatchChunk c) {
    const BatchMember& e = c.mem[blockIdx.x];
    scan_bsum_body(e.s, e.p, scan_blocks(e.m.nc));
}
__global__ void k_scan_apply_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_SCAN], c.n);
    scan_apply_body(c.mem[i].m, c.mem[i].s, member_blk(c.off[BCL_SCAN], i));
}
__global__ void k_cell_update_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_CELLS], c.n);
    cell_update_body(c.mem[i].m, c.mem[i].s, c.mem[i].p, c.mem[i].b.cell, member_blk(c.off[BCL_CELLS], i));
}
__global__ void k_wave_update_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_CELLS], c.n);
    wave_update_body(c.mem[i].m, c.mem[i].s, member_blk(c.off[BCL_CELLS], i));
}

// Time average W-bar = sum dt^n W^n / sum dt^n (Sec. 2.4 (c)).
__global__ void k_wbar(DevMesh m, DevState s, double* out) {
    const long long n = 5LL * m.nc;
    const double T = s.tsum[0];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = s.wsum[i] / T;
}

// Kn_GLL = l |grad rho| / rho with the unlimited least-squares gradient of rho
// and the VHS mean free path l = 2(5-2w)(7-2w)/15 mu / (rho sqrt(2 pi R T)).
__global__ void k_kn_gll(DevMesh m, DevState s, DevParams p, double* out) {
    const int nc = m.nc;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double rho = s.W[i];
    const int own = m.cfs[i];
    double g[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 4; ++k) {
        const int f = m.cf[k * nc + i];
        const int o = ((own >> k) & 1) ? m.f_nbr[f] : m.f_own[f];
        double v = rho;
        if (o >= 0) v = s.W[o];
        else if (p.bc[m.bf_tag[-1 - o]].type == UGKWP_BC_FARFIELD) v = p.bc[m.bf_tag[-1 - o]].W_in[0];
        for (int d = 0; d < 3; ++d) g[d] += m.lsq_c[(size_t)(3 * k + d) * nc + i] * (v - rho);
    }
    const double Ux = s.W[nc + i] / rho, Uy = s.W[2 * nc + i] / rho, Uz = s.W[3 * nc + i] / rho;
    const double pr = (s.W[4 * nc + i] - 0.5 * (rho * ((Ux * Ux + Uy * Uy) + Uz * Uz))) / (1.5 + 0.5 * (double)p.K);
    const double T = pr / (rho * p.R);
    const double mu = p.mu_ref * dm::d_exp(p.omega * dm::d_log(T / p.T_ref));
    const double w = p.omega;
    const double l = (2.0 * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / 15.0) * mu / (rho * sqrt(2.0 * 3.141592653589793 * p.R * T));
    out[i] = l * sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) / rho;
}

// The survivors' count and fixed-point mass per cell of an imported buffer.
// Imported particles mostly come sorted by cell, so each warp sums over runs
// of equal cells in its 32 slots and adds once per run (integer sums: the
// result does not depend on how they are grouped).
template <class Real>
__global__ void k_rebuild(DevMesh m, DevState s, DevParams p, PartBufRaw a) {
    const long long n = s.cnt64[CNT_N_A];
    const int32_t* cell = a.cell;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // warp-uniform bounds: every lane takes part in the run sums
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const long long i = base + lane;
        int c = -1;
        long long q = 0;
        if (i < n) {
            c = cell[i];
            if (c >= 0) q = __double2ll_rn(a.m[i] * p.qinv[0]);
        }
        const int prev = __shfl_up_sync(FULL, c, 1);
        const unsigned heads = __ballot_sync(FULL, lane == 0 || prev != c);
        const int start = 31 - __clz(heads & (FULL >> (31 - lane)));
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long o = __shfl_up_sync(FULL, q, d);
            if (lane - d >= start) q += o;
        }
        const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
        if (tail && c >= 0) {
            atomicAdd(&s.nleft[c], lane - start + 1);
            atomicAdd(reinterpret_cast<unsigned long long*>(&s.smass[c]), (unsigned long long)q);
        }
    }
}

// A state image's particles, checked and brought into the particle
// precision in the spare buffer b (its cell, m and id arrays already hold the
// image's; so do x, u and e when they come in the particle precision).
// CONVERT (mixed mode, binary64 image): x, u and e come in binary64 (staged
// [3][n], [3][n], [n]); a position becomes its offset from the anchor of its
// tet, which must be exact in binary32 and give back the position when added
// to the anchor, and the velocity and internal energy must be binary32
// values.  *err receives the smallest i << 3 | kind over the particles that
// fail, kind being the first failed check of particle i: 1 cell outside
// [0, nc), 2 internal energy negative or not a number, 3 internal energy not
// a binary32 value, 4 position or velocity not representable.
template <class Real, bool CONVERT>
__global__ void k_import(int nc, long long n, const double* anc, const double* xs, const double* us,
                         const double* es, PartBufRaw b, unsigned long long* err) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int c = b.cell[i];
        unsigned kind = 0;
        if (c < 0 || c >= nc) {
            kind = 1;
        } else if constexpr (CONVERT) {
            if (es) {
                const double ev = es[i];
                const float ef = __double2float_rn(ev);
                if (!(ev >= 0.0)) kind = 2;
                else if ((double)ef != ev) kind = 3;
                else static_cast<float*>(b.e)[i] = ef;
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double xv = xs[(size_t)d * n + i], uv = us[(size_t)d * n + i];
                const double A = anc[3 * (size_t)c + d];
                const double xl = xv - A;
                const float xf = __double2float_rn(xl), uf = __double2float_rn(uv);
                if (kind == 0 && ((double)xf != xl || A + xl != xv || (double)uf != uv)) kind = 4;
                static_cast<float*>(b.x[d])[i] = xf;
                static_cast<float*>(b.u[d])[i] = uf;
            }
        } else {
            if (b.e && !(static_cast<const Real*>(b.e)[i] >= (Real)0)) kind = 2;
        }
        if (kind) atomicMin(err, ((unsigned long long)i << 3) | kind);
    }
}

template <class Real>
__global__ void k_wp_acc(DevMesh m, DevState s, DevParams p, PartBufRaw a) {
    const long long n = s.cnt64[CNT_N_A];
    const int nc = m.nc;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const Real* ux = (const Real*)a.u[0];
    const Real* uy = (const Real*)a.u[1];
    const Real* uz = (const Real*)a.u[2];
    const Real* ei = (const Real*)a.e;  // internal energy (K > 0)
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int c = a.cell[i];
        if (c < 0) continue;
        const double u0 = (double)ux[i], u1 = (double)uy[i], u2 = (double)uz[i], mm = a.m[i];
        const double e = ei ? (double)ei[i] : 0.0;
        const double phi[5] = {mm, mm * u0, mm * u1, mm * u2, 0.5 * (mm * (((u0 * u0 + u1 * u1) + u2 * u2) + e))};
#pragma unroll
        for (int q = 0; q < 5; ++q)
            atomicAdd(reinterpret_cast<unsigned long long*>(&s.wacc[(size_t)q * nc + c]),
                      (unsigned long long)__double2ll_rn(phi[q] * p.qinv[q]));
    }
}

__global__ void k_zero_wacc(DevMesh m, DevState s) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 5LL * m.nc; i += stride) s.wacc[i] = 0;
}

// which: 1 = W^p, 2 = W^h = W - W^p
__global__ void k_wp_out(DevMesh m, DevState s, DevParams p, int which, double* out) {
    const int nc = m.nc;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double wp = ((double)s.wacc[(size_t)q * nc + i] * p.qscale[q]) / m.vol[i];
        out[(size_t)q * nc + i] = which == 1 ? wp : s.W[(size_t)q * nc + i] - wp;
    }
}

__global__ void k_prim_out(DevMesh m, DevState s, DevParams p, double* out) {
    const int nc = m.nc;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double rho = s.W[i];
    const double Ux = s.W[nc + i] / rho, Uy = s.W[2 * nc + i] / rho, Uz = s.W[3 * nc + i] / rho;
    const double U2 = (Ux * Ux + Uy * Uy) + Uz * Uz;
    const double pr = (s.W[4 * nc + i] - 0.5 * (rho * U2)) / (1.5 + 0.5 * (double)p.K);
    out[i] = rho;
    out[nc + i] = Ux;
    out[2 * nc + i] = Uy;
    out[3 * nc + i] = Uz;
    out[4 * nc + i] = pr / (rho * p.R);
}

inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

}  // namespace

int sm_count() {
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
        g = sms;
    }
    return g;
}

int particle_grid() { return sm_count() * 8; }

cudaError_t configure_cell_kernels(int carveout) {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    };
    set(k_reset);
    set(k_cell_prep);
    set(k_sample_count);
    set(k_scan_bsum);
    set(k_scan_apply);
    set(k_cell_update);
    set(k_reset_b);
    set(k_cell_prep_b);
    set(k_sample_count_b);
    set(k_scan_bsum_b);
    set(k_scan_apply_b);
    set(k_cell_update_b);
    set(k_wave_update);
    set(k_wave_update_b);
    return e;
}

void launch_reset(const DevMesh& m, const DevState& s, cudaStream_t st) {
    k_reset<<<blocks_reset(m.nc), 256, 0, st>>>(m, s);
}
void launch_cell_prep(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st) {
    k_cell_prep<<<cdiv(m.nc, 256), 256, 0, st>>>(m, s, p);
}
void launch_sample_count(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st) {
    k_sample_count<<<scan_blocks(m.nc), SCAN_BLOCK, 0, st>>>(m, s, p);
}
void launch_scan(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st) {
    k_scan_bsum<<<1, SCAN_SUM_THREADS, 0, st>>>(s, p, scan_blocks(m.nc));
    k_scan_apply<<<scan_blocks(m.nc), SCAN_BLOCK, 0, st>>>(m, s);
}
void launch_cell_update(const DevMesh& m, const DevState& s, const DevParams& p, int32_t* wcell, cudaStream_t st) {
    k_cell_update<<<cdiv(m.nc, 256), 256, 0, st>>>(m, s, p, wcell);
}
void launch_wave_update(const DevMesh& m, const DevState& s, cudaStream_t st) {
    k_wave_update<<<cdiv(m.nc, 256), 256, 0, st>>>(m, s);
}
int blocks_reset(int nc) { return cdiv(5LL * nc, 256) < 4096 ? cdiv(5LL * nc, 256) : 4096; }
int blocks_cells(int nc) { return cdiv(nc, 256); }

void launch_reset_batch(const BatchChunk& c, int blocks, cudaStream_t st) { k_reset_b<<<blocks, 256, 0, st>>>(c); }
void launch_cell_prep_batch(const BatchChunk& c, int blocks, cudaStream_t st) {
    k_cell_prep_b<<<blocks, 256, 0, st>>>(c);
}
void launch_sample_count_batch(const BatchChunk& c, int blocks, cudaStream_t st) {
    k_sample_count_b<<<blocks, SCAN_BLOCK, 0, st>>>(c);
}
void launch_scan_batch(const BatchChunk& c, int blocks, cudaStream_t st) {
    k_scan_bsum_b<<<c.n, SCAN_SUM_THREADS, 0, st>>>(c);
    k_scan_apply_b<<<blocks, SCAN_BLOCK, 0, st>>>(c);
}
void launch_cell_update_batch(const BatchChunk& c, int blocks, cudaStream_t st) {
    k_cell_update_b<<<blocks, 256, 0, st>>>(c);
}
void launch_wave_update_batch(const BatchChunk& c, int blocks, cudaStream_t st) {
    k_wave_update_b<<<blocks, 256, 0, st>>>(c);
}
void launch_rebuild_survivors(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& a,
                              cudaStream_t st) {
    if (p.precision == UGKWP_MIXED) k_rebuild<float><<<particle_grid(), 256, 0, st>>>(m, s, p, a);
    else k_rebuild<double><<<particle_grid(), 256, 0, st>>>(m, s, p, a);
}
void launch_import(int nc, long long n, bool mixed, bool convert, const double* anc, const double* xs,
                   const double* us, const double* es, const PartBufRaw& b, unsigned long long* err,
                   cudaStream_t st) {
    if (n <= 0) return;
    if (mixed && convert) k_import<float, true><<<particle_grid(), 256, 0, st>>>(nc, n, anc, xs, us, es, b, err);
    else if (mixed) k_import<float, false><<<particle_grid(), 256, 0, st>>>(nc, n, anc, xs, us, es, b, err);
    else k_import<double, false><<<particle_grid(), 256, 0, st>>>(nc, n, anc, xs, us, es, b, err);
}
void launch_wp_moments(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& a,
                       double* out, cudaStream_t st) {
    k_zero_wacc<<<cdiv(5LL * m.nc, 256), 256, 0, st>>>(m, s);
    if (p.precision == UGKWP_MIXED) k_wp_acc<float><<<particle_grid(), 256, 0, st>>>(m, s, p, a);
    else k_wp_acc<double><<<particle_grid(), 256, 0, st>>>(m, s, p, a);
    (void)out;
}
void launch_wbar(const DevMesh& m, const DevState& s, double* out, cudaStream_t st) {
    k_wbar<<<cdiv(5LL * m.nc, 256) < 4096 ? cdiv(5LL * m.nc, 256) : 4096, 256, 0, st>>>(m, s, out);
}
void launch_kn_gll(const DevMesh& m, const DevState& s, const DevParams& p, double* out, cudaStream_t st) {
    k_kn_gll<<<cdiv(m.nc, 256), 256, 0, st>>>(m, s, p, out);
}
void launch_prim_moments(const DevMesh& m, const DevState& s, const DevParams& p, int which, double* out,
                         cudaStream_t st) {
    if (which == UGKWP_PRIM) k_prim_out<<<cdiv(m.nc, 256), 256, 0, st>>>(m, s, p, out);
    else k_wp_out<<<cdiv(m.nc, 256), 256, 0, st>>>(m, s, p, which, out);
}

}  // namespace ugkwp
