// Particle kernels of the UGKWP step, templated on the particle precision
// (double: FP64 mode; float: MIXED mode).  Compiled with --fmad=false so that
// every particle trajectory and fixed-point flux is reproducible bit for bit.
//
//   k_sample_write  a5: N_sam hydro particles per cell, in pairs U +/- sqrt(RT) X
//                   with X ~ N(0, I) (Box-Muller), uniform in the tet.
//   k_sort          a11: the survivors of the last step, compacted, sorted by
//                   cell (counting sort on the scanned per-cell counts) into
//                   the working buffer, where each cell's samples follow them.
//   k_track         a6-a9: t_f = min(-tau ln eta, dt), face-by-face streaming
//                   of the cell-sorted particles, boundary interaction,
//                   particle flux (movers listed for k_movers), removal; the
//                   survivors are written compacted into the survivor buffer
//                   (block-level slot reservation).  Blocks take tiles of
//                   128 or 256 particles from a global counter.
#include "dmath.cuh"
#include "ugkwp_internal.hpp"

namespace ugkwp {

namespace {

constexpr unsigned FULL = 0xffffffffu;

enum : unsigned long long { TAG_TF = 1, TAG_SVEL = 2, TAG_SPOS = 3, TAG_WALL = 4, TAG_GP = 5, TAG_SINT = 6, TAG_WINT = 7 };

__device__ __forceinline__ void set_err(const DevState& s, int32_t bits) {
    atomicOr(reinterpret_cast<unsigned long long*>(&s.cnt64[CNT_ERR]), (unsigned long long)bits);
}

__device__ __forceinline__ unsigned long long make_id(long long step, int cell, int k) {
    return ((unsigned long long)step << 40) | ((unsigned long long)cell << 16) | (unsigned long long)k;
}

template <class Real> __device__ __forceinline__ PartView<Real> view(const PartBufRaw& r) {
    PartView<Real> v;
    for (int c = 0; c < 3; ++c) {
        v.x[c] = (Real*)r.x[c];
        v.u[c] = (Real*)r.u[c];
    }
    v.m = r.m;
    v.cell = r.cell;
    v.id = r.id;
    v.e = (Real*)r.e;
    v.e2 = (Real*)r.e2;
    return v;
}

// ------------------------------------------------------------------ sampling
// The three normals X of the pair whose first member has id `ida`: Box-Muller
// in the particle precision (binary32 in the mixed mode).
template <class Real>
__device__ __forceinline__ void pair_normals(unsigned long long ida, long long step, unsigned long long seed, Real X[3]) {
    const dm::U4 r = dm::philox(ida, (unsigned long long)step, TAG_SVEL, 0ULL, seed, 0ULL);
    if constexpr (sizeof(Real) == 4) {
        float sn, cs;
        float rad = sqrtf(-2.0f * dm::f_log(dm::u01f(r.a)));
        dm::f_sincos2pi(dm::u01f(r.b), &sn, &cs);
        X[0] = rad * cs;
        X[1] = rad * sn;
        rad = sqrtf(-2.0f * dm::f_log(dm::u01f(r.c)));
        dm::f_sincos2pi(dm::u01f(r.d), &sn, &cs);
        X[2] = rad * cs;
    } else {
        double sn, cs;
        double rad = sqrt(-2.0 * dm::d_log(dm::u01d(r.a)));
        dm::d_sincos2pi(dm::u01d(r.b), &sn, &cs);
        X[0] = rad * cs;
        X[1] = rad * sn;
        rad = sqrt(-2.0 * dm::d_log(dm::u01d(r.c)));
        dm::d_sincos2pi(dm::u01d(r.d), &sn, &cs);
        X[2] = rad * cs;
    }
}

// Internal energy of a particle with K internal degrees of freedom at spread
// sig = sqrt(RT): e = sum_{i<K} (sig N_i)^2, the normals by Box-Muller from
// Philox counters (id, step, tag, idx0 + j), four per counter, summed in
// order in the particle precision.
template <class Real>
__device__ __forceinline__ Real internal_energy(unsigned long long id, long long step, unsigned long long tag,
                                                unsigned long long idx0, int K, Real sig, unsigned long long seed) {
    Real e = (Real)0;
    for (int j = 0; 4 * j < K; ++j) {
        const dm::U4 r = dm::philox(id, (unsigned long long)step, tag, idx0 + (unsigned long long)j, seed, 0ULL);
        Real N[4];
        if constexpr (sizeof(Real) == 4) {
            float sn, cs;
            float rad = sqrtf(-2.0f * dm::f_log(dm::u01f(r.a)));
            dm::f_sincos2pi(dm::u01f(r.b), &sn, &cs);
            N[0] = rad * cs;
            N[1] = rad * sn;
            rad = sqrtf(-2.0f * dm::f_log(dm::u01f(r.c)));
            dm::f_sincos2pi(dm::u01f(r.d), &sn, &cs);
            N[2] = rad * cs;
            N[3] = rad * sn;
        } else {
            double sn, cs;
            double rad = sqrt(-2.0 * dm::d_log(dm::u01d(r.a)));
            dm::d_sincos2pi(dm::u01d(r.b), &sn, &cs);
            N[0] = rad * cs;
            N[1] = rad * sn;
            rad = sqrt(-2.0 * dm::d_log(dm::u01d(r.c)));
            dm::d_sincos2pi(dm::u01d(r.d), &sn, &cs);
            N[2] = rad * cs;
            N[3] = rad * sn;
        }
        for (int i = 0; i < 4 && 4 * j + i < K; ++i) {
            const Real si = sig * N[i];
            e = e + si * si;
        }
    }
    return e;
}

// First-order g_p sampling: X ~ N(0, I) (1 + phi(X)) for particle `id` by
// acceptance-rejection in the particle precision: attempt k draws three normals
// by Box-Muller from Philox counter (id, step, TAG_GP, 2k) and eta from
// (id, step, TAG_GP, 2k + 1); accepted if eta M <= 1 + phi(X), the last draw
// kept after GP_ATTEMPTS attempts.  Coefficients: the cell's GP_NC values.
template <class Real>
__device__ __forceinline__ void gp_normals(const double* gpc, int nc, int cell, unsigned long long id, long long step,
                                           unsigned long long seed, Real X[3]) {
    Real c[GP_NC];
#pragma unroll
    for (int k = 0; k < GP_NC; ++k) c[k] = (Real)gpc[(size_t)k * nc + cell];
    X[0] = X[1] = X[2] = (Real)0;
    for (int k = 0; k < GP_ATTEMPTS; ++k) {
        const dm::U4 r = dm::philox(id, (unsigned long long)step, TAG_GP, (unsigned long long)(2 * k), seed, 0ULL);
        const dm::U4 r2 = dm::philox(id, (unsigned long long)step, TAG_GP, (unsigned long long)(2 * k + 1), seed, 0ULL);
        Real eta;
        if constexpr (sizeof(Real) == 4) {
            float sn, cs;
            float rad = sqrtf(-2.0f * dm::f_log(dm::u01f(r.a)));
            dm::f_sincos2pi(dm::u01f(r.b), &sn, &cs);
            X[0] = rad * cs;
            X[1] = rad * sn;
            rad = sqrtf(-2.0f * dm::f_log(dm::u01f(r.c)));
            dm::f_sincos2pi(dm::u01f(r.d), &sn, &cs);
            X[2] = rad * cs;
            eta = dm::u01f(r2.a);
        } else {
            double sn, cs;
            double rad = sqrt(-2.0 * dm::d_log(dm::u01d(r.a)));
            dm::d_sincos2pi(dm::u01d(r.b), &sn, &cs);
            X[0] = rad * cs;
            X[1] = rad * sn;
            rad = sqrt(-2.0 * dm::d_log(dm::u01d(r.c)));
            dm::d_sincos2pi(dm::u01d(r.d), &sn, &cs);
            X[2] = rad * cs;
            eta = dm::u01d(r2.a);
        }
        // phi = a0 + L.X + X^T Q X + (C.X) |X|^2, in this order
        const Real lin = (c[1] * X[0] + c[2] * X[1]) + c[3] * X[2];
        const Real qd = ((c[4] * X[0]) * X[0] + (c[5] * X[1]) * X[1]) + (c[6] * X[2]) * X[2];
        const Real qo = ((c[7] * X[0]) * X[1] + (c[8] * X[0]) * X[2]) + (c[9] * X[1]) * X[2];
        const Real cub = ((c[10] * X[0] + c[11] * X[1]) + c[12] * X[2]) * ((X[0] * X[0] + X[1] * X[1]) + X[2] * X[2]);
        const Real phi = ((c[0] + lin) + (qd + (qo + qo))) + cub;
        if (eta * c[13] <= (Real)1 + phi) break;
    }
}

// Energy-matched sampling: one factor per cell, s^2 sum_j |X_j|^2 = 3 N_sam / 2,
// so the pairs' thermal energy is exactly rho^hp |Omega| (3/2) R T.  The sum
// runs over the cell's pairs in order in binary64; spread = s sqrt(RT).
template <class Real>
__global__ void __launch_bounds__(256) k_sample_scale(DevMesh m, DevState s, DevParams p) {
    const int nc = m.nc;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= nc) return;
    const long long step = s.cnt64[CNT_STEP];
    const int ns = s.nsam[cell];
    double sig = sqrt(p.R * s.prim[4 * nc + cell]);
    if (ns >= 2) {
        double S = 0.0;
        for (int j = 0; j < ns / 2; ++j) {
            Real X[3];
            pair_normals<Real>(make_id(step, cell, 2 * j), step, p.seed, X);
            const double x0 = (double)X[0], x1 = (double)X[1], x2 = (double)X[2];
            S = S + ((x0 * x0 + x1 * x1) + x2 * x2);
        }
        if (S > 0.0) sig = sig * sqrt((double)(3 * (ns / 2)) / S);
    }
    s.sig[cell] = sig;
    if constexpr (sizeof(Real) == 4) s.usig[cell].w = (float)sig;
}

template <class Real>
__global__ void __launch_bounds__(256) k_sample_write(DevMesh m, DevState s, DevParams p, PartBufRaw br) {
    if (s.cnt64[CNT_ERR] & ERRB_CAPACITY) return;
    const PartView<Real> b = view<Real>(br);
    const int nc = m.nc;
    const long long total = s.cnt64[CNT_NSAM];
    const long long step = s.cnt64[CNT_STEP];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        // owning cell: the last c with soff[c] <= g (cells with N_sam = 0 share
        // the offset of the next cell and are never the last such c)
        int lo = 0, hi = nc;  // invariant: soff[lo] <= g < soff[hi] (soff[nc] = +inf)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s.soff[mid] <= g) lo = mid; else hi = mid;
        }
        const int cell = lo;
        const int k = (int)(g - s.soff[cell]);
        const int side = k & 1;
        // the samples follow the current buffer's survivor slots, in cell order
        const long long j = s.cnt64[CNT_N_A] + g;
        if constexpr (sizeof(Real) == 4) {
            // mixed mode: binary32 arithmetic from U, sqrt(RT) and the tet's
            // vertex and edges rounded to binary32
            const float4 us = s.usig[cell];
            const unsigned long long ida = make_id(step, cell, k - side);
            const unsigned long long id = ida + (unsigned long long)side;
            const bool gp = p.sampling == UGKWP_SAMPLE_GP1;
            float X[3];
            if (gp) gp_normals<float>(s.gpc, nc, cell, id, step, p.seed, X);  // every particle on its own
            else pair_normals<float>(ida, step, p.seed, X);
            const dm::U4 rp = dm::philox(id, (unsigned long long)step, TAG_SPOS, 0ULL, p.seed, 0ULL);
            float a = dm::u01f(rp.a), bb = dm::u01f(rp.b), cc = dm::u01f(rp.c);
            if (a + bb > 1.0f) { a = 1.0f - a; bb = 1.0f - bb; }
            if (bb + cc > 1.0f) {
                const float t = cc;
                cc = 1.0f - a - bb;
                bb = 1.0f - t;
            } else if (a + bb + cc > 1.0f) {
                const float t = cc;
                cc = a + bb + cc - 1.0f;
                a = 1.0f - bb - t;
            }
            const float U[3] = {us.x, us.y, us.z};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float P0 = m.vtx_f[(size_t)c * nc + cell];
                const float E1 = m.vtx_f[(size_t)(3 + c) * nc + cell];
                const float E2 = m.vtx_f[(size_t)(6 + c) * nc + cell];
                const float E3 = m.vtx_f[(size_t)(9 + c) * nc + cell];
                b.x[c][j] = P0 + ((a * E1 + bb * E2) + cc * E3);
                b.u[c][j] = (gp || side == 0) ? U[c] + us.w * X[c] : U[c] - us.w * X[c];
            }
            b.m[j] = s.msam[cell];
            b.cell[j] = cell;
            b.id[j] = id;
            if (p.K > 0) b.e[j] = internal_energy<float>(id, step, TAG_SINT, 0ULL, p.K, us.w, p.seed);
            continue;
        }
        const double U[3] = {s.prim[nc + cell], s.prim[2 * nc + cell], s.prim[3 * nc + cell]};
        const double sig = p.sampling == UGKWP_SAMPLE_ENERGY_MATCHED ? s.sig[cell] : sqrt(p.R * s.prim[4 * nc + cell]);
        const unsigned long long ida = make_id(step, cell, k - side);
        const unsigned long long id = ida + (unsigned long long)side;
        const bool gp = p.sampling == UGKWP_SAMPLE_GP1;
        double X[3];
        if (gp) gp_normals<double>(s.gpc, nc, cell, id, step, p.seed, X);
        else pair_normals<double>(ida, step, p.seed, X);
        const dm::U4 rp = dm::philox(id, (unsigned long long)step, TAG_SPOS, 0ULL, p.seed, 0ULL);
        double a = dm::u01d(rp.a), bb = dm::u01d(rp.b), cc = dm::u01d(rp.c);
        // cube -> prism -> tet folding of a uniform point (Rocchini & Cignoni 2000)
        if (a + bb > 1.0) { a = 1.0 - a; bb = 1.0 - bb; }
        if (bb + cc > 1.0) {
            const double t = cc;
            cc = 1.0 - a - bb;
            bb = 1.0 - t;
        } else if (a + bb + cc > 1.0) {
            const double t = cc;
            cc = a + bb + cc - 1.0;
            a = 1.0 - bb - t;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double P0 = m.vtx[(size_t)c * nc + cell];
            const double E1 = m.vtx[(size_t)(3 + c) * nc + cell] - P0;
            const double E2 = m.vtx[(size_t)(6 + c) * nc + cell] - P0;
            const double E3 = m.vtx[(size_t)(9 + c) * nc + cell] - P0;
            b.x[c][j] = (Real)(P0 + ((a * E1 + bb * E2) + cc * E3));
            b.u[c][j] = (Real)((gp || side == 0) ? U[c] + sig * X[c] : U[c] - sig * X[c]);
        }
        b.m[j] = s.msam[cell];
        b.cell[j] = cell;
        b.id[j] = id;
        if (p.K > 0) b.e[j] = (Real)internal_energy<double>(id, step, TAG_SINT, 0ULL, p.K, sig, p.seed);
    }
}

// ------------------------------------------------------------------ tracking
template <class Real> struct Trk;
template <> struct Trk<float> {
    __device__ static __forceinline__ void plane(const DevMesh& m, int tet, int k, float& nx, float& ny, float& nz,
                                                 float& d) {
        const float4 v = m.trk_f[tet].pl[k];
        nx = v.x; ny = v.y; nz = v.z; d = v.w;
    }
    __device__ static __forceinline__ int4 nbv(const DevMesh& m, int tet) { return m.trk_f[tet].nb; }
    __device__ static __forceinline__ float tau(const DevState& s, int c) { return s.tauf[c]; }
    __device__ static __forceinline__ float tf(float tau, unsigned long long r) {
        return -(tau * dm::f_log(dm::u01f(r)));
    }
};
template <> struct Trk<double> {
    __device__ static __forceinline__ void plane(const DevMesh& m, int tet, int k, double& nx, double& ny,
                                                 double& nz, double& d) {
        const Dbl4 v = m.trk_d[tet].pl[k];
        nx = v.x; ny = v.y; nz = v.z; d = v.w;
    }
    __device__ static __forceinline__ int4 nbv(const DevMesh& m, int tet) { return m.trk_d[tet].nb; }
    __device__ static __forceinline__ double tau(const DevState& s, int c) { return s.tau[c]; }
    __device__ static __forceinline__ double tf(double tau, unsigned long long r) {
        return -(tau * dm::d_log(dm::u01d(r)));
    }
};

// Round-to-nearest-even of v 2^-e for a binary64 v, from the bits of v with
// integer operations only (v 2^-e is an exact exponent shift, so this equals
// rounding the scaled binary64 value); false (q = 0) if v is not finite or
// |v 2^-e| >= 2^62.  Keeps the conversions off the FP64 pipe.
__device__ __forceinline__ bool fixed_of(double v, int e, long long& q) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & 0x000fffffffffffffULL;
    q = 0;
    if (ex == 0x7ff) return false;
    int sh;  // |v| 2^-e = mant 2^sh
    if (ex == 0) {
        sh = 1 - 1075 - e;
    } else {
        mant |= 0x0010000000000000ULL;
        sh = ex - 1075 - e;
    }
    unsigned long long mag;
    if (sh >= 0) {
        if (mant == 0) return true;
        if (sh > 9) return false;  // mant >= 2^52 when nonzero and normal: 2^(52+10) = 2^62
        mag = mant << sh;
        if (mag >= (1ULL << 62)) return false;
    } else {
        const int r = -sh;
        if (r > 63) return true;
        const unsigned long long hi = mant >> r;
        const unsigned long long rem = mant & ((1ULL << r) - 1ULL);
        const unsigned long long half = 1ULL << (r - 1);
        mag = hi + ((rem > half || (rem == half && (hi & 1ULL))) ? 1ULL : 0ULL);
    }
    q = (bits >> 63) ? -(long long)mag : (long long)mag;
    return true;
}

// Exact binary32 -> binary64 widening on the bits (integer pipes only).
__device__ __forceinline__ double widen(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    int ex = (int)((b >> 23) & 0xff);
    unsigned mant = b & 0x7fffffu;
    if (ex == 0xff) return __longlong_as_double((long long)(sign | (0x7ffULL << 52) | ((unsigned long long)mant << 29)));
    if (ex == 0) {
        if (mant == 0) return __longlong_as_double((long long)sign);
        const int k = __clz(mant) - 8;  // shift that brings the leading one to bit 23
        mant = (mant << k) & 0x7fffffu;
        ex = 1 - k;
    }
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(ex - 127 + 1023) << 52) | ((unsigned long long)mant << 29)));
}
__device__ __forceinline__ double widen(double d) { return d; }

// Fixed-point image of phi = m (1, u, |u|^2/2); false if a value leaves |v| < 2^62.
// The factor 1/2 of the energy is applied as an exponent shift.
template <class Real>
__device__ __forceinline__ bool phi_q(const Real* u, Real e, double mm, const DevParams& p, long long q[5]) {
    const double u0 = widen(u[0]), u1 = widen(u[1]), u2 = widen(u[2]);
    bool ok = fixed_of(mm, p.exps[0], q[0]);
    ok &= fixed_of(mm * u0, p.exps[1], q[1]);
    ok &= fixed_of(mm * u1, p.exps[2], q[2]);
    ok &= fixed_of(mm * u2, p.exps[3], q[3]);
    ok &= fixed_of(mm * (((u0 * u0 + u1 * u1) + u2 * u2) + widen(e)), p.exps[4] + 1, q[4]);
    return ok;
}

// round-to-nearest-even of m 2^-e for a finite m >= 0, computed on the bits of
// m with integer operations only (m 2^-e is an exact exponent shift, so this
// equals rounding the binary64 product); false if the result is >= 2^62.
__device__ __forceinline__ bool fixed_of_mass(double m, int e, long long& q) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(m);
    const int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & 0x000fffffffffffffULL;
    int s;  // value = mant 2^s
    if (ex == 0) {
        s = 1 - 1075 - e;
    } else {
        mant |= 0x0010000000000000ULL;
        s = ex - 1075 - e;
    }
    if (ex == 0x7ff || (bits >> 63)) { q = 0; return false; }
    if (s >= 0) {
        if (mant == 0) { q = 0; return true; }
        if (s > 9) { q = 0; return false; }  // mant < 2^53: 2^(53+s) > 2^62
        const unsigned long long v = mant << s;
        if (v >= (1ULL << 62)) { q = 0; return false; }
        q = (long long)v;
        return true;
    }
    const int r = -s;
    if (r > 63) { q = 0; return true; }
    const unsigned long long hi = mant >> r;
    const unsigned long long rem = mant & ((1ULL << r) - 1ULL);
    const unsigned long long half = 1ULL << (r - 1);
    q = (long long)(hi + ((rem > half || (rem == half && (hi & 1ULL))) ? 1ULL : 0ULL));
    return true;
}

// ---- bulk copies of particle tiles into shared memory: the copy engine
// (cp.async.bulk, TMA) writes a stage and completes the transaction count of
// the stage's mbarrier; the block waits on the barrier's phase parity.
__device__ __forceinline__ unsigned smem_addr(const void* ptr) { return (unsigned)__cvta_generic_to_shared(ptr); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity to complete: at most MBAR_TRIES
// tests (each may suspend the thread for a while), false if it did not.
constexpr int MBAR_TRIES = 1 << 22;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (int k = 0; k < MBAR_TRIES; ++k)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// One stage of T particles in shared memory, structure of arrays like the
// particle buffer: x[3], u[3] (particle precision), e (KE), m, id, cell.  Every
// array starts on a 16-byte boundary (T RS is a multiple of 512).
template <class Real, bool KE, int T> struct Stage {
    static constexpr int RS = (int)sizeof(Real);
    static constexpr int X = 0;
    static constexpr int U = 3 * T * RS;
    static constexpr int E = 6 * T * RS;
    static constexpr int M = (KE ? 7 : 6) * T * RS;
    static constexpr int ID = M + 8 * T;
    static constexpr int CELL = ID + 8 * T;
    static constexpr int BYTES = CELL + 4 * T;
};

// Thread 0: bulk copies of the tile of T particles from index t0 (a multiple
// of T: every source starts 16-byte aligned, and the particle arrays hold
// whole tiles) into stage `st`, completing on `bar`.
template <class Real, bool KE, int T>
__device__ __forceinline__ void stage_tile(char* st, unsigned long long* bar, const PartView<Real>& b, long long t0) {
    using L = Stage<Real, KE, T>;
    mbar_expect(bar, (unsigned)L::BYTES);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        bulk_load(st + L::X + c * T * L::RS, b.x[c] + t0, T * L::RS, bar);
        bulk_load(st + L::U + c * T * L::RS, b.u[c] + t0, T * L::RS, bar);
    }
    if constexpr (KE) bulk_load(st + L::E, b.e + t0, T * L::RS, bar);
    bulk_load(st + L::M, b.m + t0, 8 * T, bar);
    bulk_load(st + L::ID, b.id + t0, 8 * T, bar);
    bulk_load(st + L::CELL, b.cell + t0, 4 * T, bar);
}

// Thread 0's source of tiles: grabs of TILE_GRAB consecutive tiles from the
// global counter (one atomic per grab), handed out in order, so the tiles a
// block walks increase.  Returns the first particle index of the next tile.
struct TileQueue {
    long long next = 0, end = 0;
};
__device__ __forceinline__ long long next_tile(TileQueue& q, int64_t* ctr, int T) {
    if (q.next == q.end) {
        q.next = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(ctr), 1ULL) * TILE_GRAB;
        q.end = q.next + TILE_GRAB;
    }
    return (q.next++) * T;
}

// KE: the particles carry an internal energy (K > 0).  THREADS: particles per
// tile (one per thread).  STAGES = 0: each thread loads its particle from the
// buffer when its tile starts; STAGES > 0: the tiles are staged in shared
// memory by bulk copies, STAGES - 1 tiles ahead of the one being walked.
template <class Real, bool KE, int THREADS, int STAGES>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_track(DevMesh m, DevState s, DevParams p, PartBufRaw br,
                                                                  PartBufRaw nr, PartBufRaw ar) {
    constexpr int NW = THREADS / 32;
    using L = Stage<Real, KE, THREADS>;
    if (s.cnt64[CNT_ERR] & ERRB_CAPACITY) return;
    const PartView<Real> b = view<Real>(br);   // this step's particles: survivors, then samples
    const PartView<Real> nxt = view<Real>(nr);  // the next step's survivors, compacted
    const PartView<Real> mv = view<Real>(ar);  // mover list: x = u at start, u = u at end
    const long long n = s.cnt64[CNT_N_B];
    const long long step = s.cnt64[CNT_STEP];
    const double dt = s.dt[0];
    const Real dtR = (Real)dt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // slot bookkeeping in two sets, alternating between tiles, so that no
    // barrier is needed after a tile's stores: a set is rewritten two tiles
    // later, after two barriers every warp has passed
    __shared__ int sh_cnt[2][NW];
    __shared__ long long sh_base[2], sh_tile[2];
    const long long wtot = s.cnt64[CNT_WTOT];  // overflow slots start after the buckets
    int par = 0;
    __shared__ unsigned long long sh_red[NW][8];
    // staged tiles: first particle index per stage, one mbarrier per stage
    extern __shared__ __align__(16) char stg[];
    __shared__ unsigned long long sh_bar[STAGES > 0 ? STAGES : 1];
    __shared__ long long sh_stile[STAGES > 0 ? STAGES : 1];
    // per-thread counters, reduced once per block at the end
    unsigned c_valid = 0, c_coll = 0, c_exit = 0, c_lost = 0, c_cross = 0, c_wall = 0, c_surv = 0;
    // tiles of THREADS particles are taken from a global counter, so that
    // blocks that start late (or walk short paths) take fewer tiles
    TileQueue tq;  // thread 0's
    if (threadIdx.x == 0) {
        if constexpr (STAGES > 0) {
            for (int k = 0; k < STAGES; ++k) mbar_init(&sh_bar[k]);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            for (int k = 0; k < STAGES; ++k) {
                const long long t0 = next_tile(tq, &s.cnt64[CNT_TILE], THREADS);
                sh_stile[k] = t0;
                if (t0 < n) stage_tile<Real, KE, THREADS>(stg + k * L::BYTES, &sh_bar[k], b, t0);
            }
        } else {
            sh_tile[0] = next_tile(tq, &s.cnt64[CNT_TILE], THREADS);
        }
    }
    __syncthreads();
    int slot = 0;        // stage of this tile
    unsigned phase = 0;  // parity of the stage's mbarrier phase this tile completes
    for (;;) {
        const long long bb = STAGES > 0 ? sh_stile[slot] : sh_tile[par];  // block-uniform
        if (bb >= n) break;
        const long long i = bb + threadIdx.x;
        // a stage whose copies did not complete within the wait's limit is
        // not read; the block stops at the next barrier
        const bool staged = STAGES == 0 || mbar_wait(&sh_bar[slot], phase);
        // the slot's start cell; -1 marks a hole of a survivor bucket
        int c0 = -1, tet = -1;
        if (i < n && staged)
            c0 = STAGES > 0 ? reinterpret_cast<const int*>(stg + slot * L::BYTES + L::CELL)[threadIdx.x] : b.cell[i];
        const bool valid = c0 >= 0;
        int status = 0, ncross = 0, nrefl = 0, nwall = 0;
        long long qmass = 0;
        bool survivor = false, mover = false, exited = false;
        Real us[3] = {(Real)0, (Real)0, (Real)0}, ue[3] = {(Real)0, (Real)0, (Real)0};
        Real xe[3] = {(Real)0, (Real)0, (Real)0};
        Real es = (Real)0, ee = (Real)0;  // internal energy at start and end (KE)
        double mm = 0.0;
        unsigned long long id = 0;
        if (valid) {
            Real x0[3], u[3];
            if constexpr (STAGES > 0) {
                const char* st = stg + slot * L::BYTES;
                const int k = threadIdx.x;
                id = reinterpret_cast<const unsigned long long*>(st + L::ID)[k];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    x0[c] = reinterpret_cast<const Real*>(st + L::X + c * THREADS * L::RS)[k];
                    u[c] = reinterpret_cast<const Real*>(st + L::U + c * THREADS * L::RS)[k];
                }
                mm = reinterpret_cast<const double*>(st + L::M)[k];
                if constexpr (KE) {
                    es = reinterpret_cast<const Real*>(st + L::E)[k];
                    ee = es;
                }
            } else {
                id = b.id[i];
#pragma unroll
                for (int c = 0; c < 3; ++c) { x0[c] = b.x[c][i]; u[c] = b.u[c][i]; }
                mm = b.m[i];
                if constexpr (KE) {
                    es = b.e[i];
                    ee = es;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) us[c] = u[c];
            Real t_end = dtR;
            bool coll = false;
            if ((long long)(id >> 40) != step) {
                // Philox4x32-10, counter (id low, id high, step, TAG_TF), key (seed low, seed high)
                const unsigned long long r = dm::philox32_2((unsigned)id, (unsigned)(id >> 32), (unsigned)step,
                                                            (unsigned)TAG_TF, (unsigned)p.seed,
                                                            (unsigned)(p.seed >> 32));
                const Real tf = Trk<Real>::tf(Trk<Real>::tau(s, c0), r);
                if (tf < dtR) { coll = true; t_end = tf; }
            }
            // ---- face-by-face walk along x0 + u (t - t0)
            tet = c0;
            int last = -1;
            Real t0 = (Real)0;
            for (;;) {
                // the tet's neighbour codes, loaded with its planes (they sit in
                // another sector of the tet's record)
                const int4 nbv = Trk<Real>::nbv(m, tet);
                // smallest crossing time (d - n.x0)/(u.n) over u.n > 0, compared
                // by cross products (positive denominators), one division
                int best = -1;
                Real nbest = (Real)0, dbest = (Real)1;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k == last) continue;
                    Real nx, ny, nz, d;
                    Trk<Real>::plane(m, tet, k, nx, ny, nz, d);
                    const Real un = (u[0] * nx + u[1] * ny) + u[2] * nz;
                    if (un > (Real)0) {
                        const Real xn = (x0[0] * nx + x0[1] * ny) + x0[2] * nz;
                        const Real num = d - xn;
                        if (best < 0 || num * dbest < nbest * un) { best = k; nbest = num; dbest = un; }
                    }
                }
                Real sbest = best >= 0 ? nbest / dbest : (Real)0;
                const Real rem = t_end - t0;
                if (best < 0 || sbest >= rem) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) xe[c] = x0[c] + u[c] * rem;
                    break;
                }
                if (sbest < (Real)0) sbest = (Real)0;
                ++ncross;
                if (ncross > p.max_crossings) {
                    status |= 4;
#pragma unroll
                    for (int c = 0; c < 3; ++c) xe[c] = x0[c];
                    break;
                }
                const int code = best == 0 ? nbv.x : best == 1 ? nbv.y : best == 2 ? nbv.z : nbv.w;
                if (code >= 0) { tet = code >> 2; last = code & 3; continue; }
                const int bi = -1 - code;
                const DevBc& bc = p.bc[m.bf_tag[bi]];
                if (bc.type == UGKWP_BC_FARFIELD || bc.type == UGKWP_BC_OUTFLOW) { status |= 2; break; }
                Real xh[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) xh[c] = x0[c] + u[c] * sbest;
                if (bc.type == UGKWP_BC_SPECULAR) {
                    Real nx, ny, nz, d;
                    Trk<Real>::plane(m, tet, best, nx, ny, nz, d);
                    const Real un = (u[0] * nx + u[1] * ny) + u[2] * nz;
                    const Real two = un + un;
                    u[0] = u[0] - two * nx;
                    u[1] = u[1] - two * ny;
                    u[2] = u[2] - two * nz;
                } else {
                    // diffuse re-emission, full accommodation: |u_n| = sqrt(-2 R T_w ln eta),
                    // tangential components U_w,t + sqrt(R T_w) N(0,1)
                    const dm::U4 r = dm::philox(id, (unsigned long long)step, TAG_WALL, (unsigned long long)nwall,
                                                p.seed, 0ULL);
                    if constexpr (sizeof(Real) == 4) {
                        // mixed mode: binary32 from the wall constants and the
                        // face frame rounded to binary32
                        const float vn = sqrtf(bc.c2rt_f * dm::f_log(dm::u01f(r.a)));
                        const float rad = sqrtf(-2.0f * dm::f_log(dm::u01f(r.b)));
                        float sn, cs;
                        dm::f_sincos2pi(dm::u01f(r.c), &sn, &cs);
                        const int nbf = m.nbf;
                        const float v1 = m.bf_f[(size_t)9 * nbf + bi] + bc.sw_f * (rad * cs);
                        const float v2 = m.bf_f[(size_t)10 * nbf + bi] + bc.sw_f * (rad * sn);
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            u[c] = ((-vn) * m.bf_f[(size_t)c * nbf + bi] + v1 * m.bf_f[(size_t)(3 + c) * nbf + bi]) +
                                   v2 * m.bf_f[(size_t)(6 + c) * nbf + bi];
                        if constexpr (KE)
                            ee = internal_energy<float>(id, step, TAG_WINT, 2ULL * (unsigned long long)nwall, p.K, bc.sw_f,
                                                        p.seed);
                    } else {
                        const double vn = sqrt(-2.0 * p.R * bc.T_w * dm::d_log(dm::u01d(r.a)));
                        const double rad = sqrt(-2.0 * dm::d_log(dm::u01d(r.b)));
                        double sn, cs;
                        dm::d_sincos2pi(dm::u01d(r.c), &sn, &cs);
                        const double sw = sqrt(p.R * bc.T_w);
                        const int nbf = m.nbf;
                        double n3[3], t1[3], t2[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            n3[c] = m.bf_n[(size_t)c * nbf + bi];
                            t1[c] = m.bf_t1[(size_t)c * nbf + bi];
                            t2[c] = m.bf_t2[(size_t)c * nbf + bi];
                        }
                        const double v1 = ((bc.U_w[0] * t1[0] + bc.U_w[1] * t1[1]) + bc.U_w[2] * t1[2]) + sw * (rad * cs);
                        const double v2 = ((bc.U_w[0] * t2[0] + bc.U_w[1] * t2[1]) + bc.U_w[2] * t2[2]) + sw * (rad * sn);
#pragma unroll
                        for (int c = 0; c < 3; ++c) u[c] = (Real)(((-vn) * n3[c] + v1 * t1[c]) + v2 * t2[c]);
                        if constexpr (KE)
                            ee = (Real)internal_energy<double>(id, step, TAG_WINT, 2ULL * (unsigned long long)nwall, p.K,
                                                               sw, p.seed);
                    }
                    ++nwall;
                }
                ++nrefl;
#pragma unroll
                for (int c = 0; c < 3; ++c) x0[c] = xh[c];
                t0 = t0 + sbest;
                last = best;
            }
            exited = status & 2;
            const bool lost = status & 4;
            survivor = !exited && (!coll || lost);
            if (coll && !lost && !exited) status |= 1;
            // ---- particle flux by counting: a particle that ends in its start
            // cell with its velocity unchanged contributes nothing; the others
            // are listed for the binary64 flux pass
            mover = exited || tet != c0 || nrefl > 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) ue[c] = u[c];
            if (survivor && !fixed_of_mass(mm, p.exps[0], qmass)) set_err(s, ERRB_FIXED_OVERFLOW);
            c_valid += 1;
            c_coll += status & 1;
            c_exit += (status >> 1) & 1;
            c_lost += (status >> 2) & 1;
            c_cross += ncross;
            c_wall += nwall;
        }
        // ---- a11: each survivor goes to the bucket of its end cell in the
        // next buffer, so the next step finds the particles sorted by cell.
        // Lanes with the same end cell take consecutive slots from the cell's
        // count (one atomic per group); the count is also the cell's survivor
        // count N_left of the next step.  A survivor beyond its bucket takes an
        // overflow slot after the buckets.
        const int key = survivor ? tet : -1;
        int srank = 0;  // the survivor's slot in its bucket, written after the movers' barriers
        {
            const unsigned peers = __match_any_sync(FULL, key);
            const int leader = __ffs(peers) - 1;
            int rank = 0;
            if (lane == leader && key >= 0) rank = atomicAdd(&s.nleft_next[key], __popc(peers));
            rank = __shfl_sync(FULL, rank, leader) + __popc(peers & ((1u << lane) - 1u));
            srank = rank;
        }
        // ---- survivors' fixed-point mass per end cell: segmented reduction
        // over lanes with equal keys in a row, one atomic per run
        {
            long long v = survivor ? qmass : 0;
            const int prev = __shfl_up_sync(FULL, key, 1);
            const bool head = lane == 0 || prev != key;
            const unsigned heads = __ballot_sync(FULL, head);
            const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long o = __shfl_up_sync(FULL, v, d);
                if (lane - d >= start) v += o;
            }
            const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
            if (tail && key >= 0) atomicAdd(reinterpret_cast<unsigned long long*>(&s.smass_next[key]), (unsigned long long)v);
        }
        c_surv += survivor ? 1u : 0u;
        // ---- movers: one slot reservation per block and iteration
        const unsigned mmask = __ballot_sync(FULL, mover);
        if (lane == 0) sh_cnt[par][warp] = __popc(mmask);
        if (__syncthreads_or(!staged)) {
            // a stage wait gave up: report it, give the copies still in flight
            // a bounded wait (shared memory must not be released under them)
            // and stop; the step's particle state is not valid
            if (threadIdx.x == 0) {
                set_err(s, ERRB_STAGE_WAIT);
                if constexpr (STAGES > 0) {
                    unsigned ph = phase;
                    for (int k = 0, sl = slot; k < STAGES; ++k) {
                        if (sh_stile[sl] < n) mbar_wait(&sh_bar[sl], ph);
                        if (++sl == STAGES) { sl = 0; ph ^= 1u; }
                    }
                }
            }
            return;
        }
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < NW; ++w) {
                const int c = sh_cnt[par][w];
                sh_cnt[par][w] = tot;
                tot += c;
            }
            sh_base[par] =
                tot ? (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&s.cnt64[CNT_RESV]), (unsigned long long)tot)
                    : 0LL;
            if constexpr (STAGES > 0) {
                // refill this tile's stage (every thread read its particle from
                // it before the barrier above) with the tile STAGES ahead
                const long long t0 = next_tile(tq, &s.cnt64[CNT_TILE], THREADS);
                sh_stile[slot] = t0;
                if (t0 < n) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    stage_tile<Real, KE, THREADS>(stg + slot * L::BYTES, &sh_bar[slot], b, t0);
                }
            } else {
                // the next tile, in the other set (its last readers read it
                // before the barrier above)
                sh_tile[par ^ 1] = next_tile(tq, &s.cnt64[CNT_TILE], THREADS);
            }
        }
        __syncthreads();
        if (survivor) {
            long long j = -1;
            if (srank < s.wcap[tet]) {
                j = (long long)s.woff[tet] + srank;
            } else {
                const long long o = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&s.cnt64[CNT_OVF]), 1ULL);
                if (o < p.capacity - wtot) j = wtot + o;
                else set_err(s, ERRB_CAPACITY);
            }
            if (j >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    nxt.x[c][j] = xe[c];
                    nxt.u[c][j] = ue[c];
                }
                nxt.m[j] = mm;
                nxt.cell[j] = tet;
                nxt.id[j] = id;
                if constexpr (KE) nxt.e[j] = ee;
            }
        }
        if (mover) {
            const long long j = sh_base[par] + sh_cnt[par][warp] + __popc(mmask & ((1u << lane) - 1u));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                mv.x[c][j] = us[c];
                mv.u[c][j] = ue[c];
            }
            mv.m[j] = mm;
            mv.cell[j] = c0;
            mv.id[j] = ((unsigned long long)(unsigned)tet << 1) | (exited ? 1ULL : 0ULL);
            if constexpr (KE) {
                mv.e[j] = es;
                mv.e2[j] = ee;
            }
        }
        par ^= 1;
        if (STAGES > 0 && ++slot == STAGES) {
            slot = 0;
            phase ^= 1u;
        }
    }
    // ---- counters: one atomic per block and counter (survivors were counted
    // by their slot reservations)
    unsigned vals[7] = {c_valid, c_coll, c_exit, c_lost, c_cross, c_wall, c_surv};
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const unsigned w = __reduce_add_sync(FULL, vals[k]);
        if (lane == 0) sh_red[warp][k] = w;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        unsigned long long t = 0;
        for (int w = 0; w < NW; ++w) t += sh_red[w][threadIdx.x];
        const int slot[7] = {CNT_TRACKED, CNT_COLLIDED, CNT_EXITED, CNT_LOST, CNT_CROSSINGS, CNT_WALL, CNT_SURV};
        if (t) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&s.cnt64[slot[threadIdx.x]]), t);
            if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&s.cnt64[CNT_MOVES]), t);
            if (threadIdx.x == 3) set_err(s, ERRB_TRACK_LIMIT);
        }
    }
}

// Counting flux of the listed movers: -phi(u_start) at the start cell and, unless
// the particle left the domain, +phi(u_end) at the end cell (full warps of
// binary64 work, kept out of the tracking kernel).
template <class Real>
__global__ void __launch_bounds__(256) k_movers(DevMesh m, DevState s, DevParams p, PartBufRaw ar) {
    if (s.cnt64[CNT_ERR] & ERRB_CAPACITY) return;
    const PartView<Real> mv = view<Real>(ar);
    const long long n = s.cnt64[CNT_RESV];
    const int nc = m.nc;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    // whole warps per iteration: the start-cell sums are reduced over runs of
    // equal start cells within the warp (the list is ordered by start cell
    // within each tracking tile), one atomic per run and quantity
    for (long long j0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < n; j0 += stride) {
        const long long j = j0 + lane;
        const bool valid = j < n;
        Real us[3] = {(Real)0, (Real)0, (Real)0}, ue[3] = {(Real)0, (Real)0, (Real)0};
        double mm = 0.0;
        int c0 = -1, c1 = -1;
        bool exited = true;
        long long q0[5] = {0, 0, 0, 0, 0}, q1[5] = {0, 0, 0, 0, 0};
        if (valid) {
#pragma unroll
            for (int c = 0; c < 3; ++c) { us[c] = mv.x[c][j]; ue[c] = mv.u[c][j]; }
            mm = mv.m[j];
            c0 = mv.cell[j];
            const unsigned long long code = mv.id[j];
            c1 = (int)(code >> 1);
            exited = code & 1ULL;
            const Real es = mv.e ? mv.e[j] : (Real)0, ee = mv.e2 ? mv.e2[j] : (Real)0;
            bool ok = phi_q(us, es, mm, p, q0);
            ok &= phi_q(ue, ee, mm, p, q1);
            if (!ok) set_err(s, ERRB_FIXED_OVERFLOW);
        }
        const int prev = __shfl_up_sync(FULL, c0, 1);
        const bool head = lane == 0 || prev != c0;
        const unsigned heads = __ballot_sync(FULL, head);
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            long long v = -q0[q];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long o = __shfl_up_sync(FULL, v, d);
                if (lane - d >= start) v += o;
            }
            if (tail && c0 >= 0)
                atomicAdd(reinterpret_cast<unsigned long long*>(&s.pflux[(size_t)q * nc + c0]), (unsigned long long)v);
        }
        if (valid && !exited) {
#pragma unroll
            for (int q = 0; q < 5; ++q)
                atomicAdd(reinterpret_cast<unsigned long long*>(&s.pflux[(size_t)q * nc + c1]), (unsigned long long)q1[q]);
        }
    }
}

}  // namespace

void launch_sample_write(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& b,
                         int blocks, cudaStream_t st) {
    (void)m;
    if (p.precision == UGKWP_MIXED) k_sample_write<float><<<blocks, 256, 0, st>>>(m, s, p, b);
    else k_sample_write<double><<<blocks, 256, 0, st>>>(m, s, p, b);
}

void launch_sample_scale(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st) {
    if (p.precision == UGKWP_MIXED) k_sample_scale<float><<<(m.nc + 255) / 256, 256, 0, st>>>(m, s, p);
    else k_sample_scale<double><<<(m.nc + 255) / 256, 256, 0, st>>>(m, s, p);
}

namespace {
template <class Real, bool KE, int T, int S>
void track_as(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& b, const PartBufRaw& nxt,
              const PartBufRaw& movers, int blocks, cudaStream_t st) {
    const int smem = S > 0 ? S * Stage<Real, KE, T>::BYTES : 0;
    k_track<Real, KE, T, S><<<blocks, T, smem, st>>>(m, s, p, b, nxt, movers);
}
template <class Real, bool KE>
void track_shape(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& b, const PartBufRaw& nxt,
                 const PartBufRaw& movers, const TrackShape& sh, int blocks, cudaStream_t st) {
    if (sh.threads == 256) {
        if (sh.stages == 2) track_as<Real, KE, 256, 2>(m, s, p, b, nxt, movers, blocks, st);
        else if (sh.stages == 3) track_as<Real, KE, 256, 3>(m, s, p, b, nxt, movers, blocks, st);
        else track_as<Real, KE, 256, 0>(m, s, p, b, nxt, movers, blocks, st);
    } else {
        if (sh.stages == 2) track_as<Real, KE, 128, 2>(m, s, p, b, nxt, movers, blocks, st);
        else if (sh.stages == 3) track_as<Real, KE, 128, 3>(m, s, p, b, nxt, movers, blocks, st);
        else track_as<Real, KE, 128, 0>(m, s, p, b, nxt, movers, blocks, st);
    }
}
}  // namespace

void launch_track(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& b, const PartBufRaw& nxt,
                  const PartBufRaw& movers, const TrackShape& sh, int blocks, cudaStream_t st) {
    if (p.precision == UGKWP_MIXED) {
        if (p.K > 0) track_shape<float, true>(m, s, p, b, nxt, movers, sh, blocks, st);
        else track_shape<float, false>(m, s, p, b, nxt, movers, sh, blocks, st);
    } else {
        if (p.K > 0) track_shape<double, true>(m, s, p, b, nxt, movers, sh, blocks, st);
        else track_shape<double, false>(m, s, p, b, nxt, movers, sh, blocks, st);
    }
}

namespace {
// Attributes of every tracking shape of one particle type: the dynamic shared
// memory its stages take, and the preferred carveout; the carveout also for
// the other particle kernels of that type.
template <class Real, bool KE> cudaError_t configure_type(int carveout) {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto f, int smem) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    };
    set(k_track<Real, KE, 128, 0>, 0);
    set(k_track<Real, KE, 128, 2>, 2 * Stage<Real, KE, 128>::BYTES);
    set(k_track<Real, KE, 128, 3>, 3 * Stage<Real, KE, 128>::BYTES);
    set(k_track<Real, KE, 256, 0>, 0);
    set(k_track<Real, KE, 256, 2>, 2 * Stage<Real, KE, 256>::BYTES);
    set(k_track<Real, KE, 256, 3>, 3 * Stage<Real, KE, 256>::BYTES);
    set(k_sample_write<Real>, 0);
    set(k_sample_scale<Real>, 0);
    set(k_movers<Real>, 0);
    return e;
}
}  // namespace

cudaError_t configure_particle_kernels(const DevParams& p, const TrackShape& sh, int carveout) {
    (void)sh;
    if (p.precision == UGKWP_MIXED) return p.K > 0 ? configure_type<float, true>(carveout) : configure_type<float, false>(carveout);
    return p.K > 0 ? configure_type<double, true>(carveout) : configure_type<double, false>(carveout);
}

int track_smem_bytes(const DevParams& p, const TrackShape& sh) {
    if (sh.stages <= 0) return 0;
    const int rs = p.precision == UGKWP_MIXED ? 4 : 8;
    const int arrays = 6 + (p.K > 0 ? 1 : 0);
    return sh.stages * sh.threads * (arrays * rs + 8 + 8 + 4);
}

void launch_movers(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& a, int blocks, cudaStream_t st) {
    if (p.precision == UGKWP_MIXED) k_movers<float><<<blocks, 256, 0, st>>>(m, s, p, a);
    else k_movers<double><<<blocks, 256, 0, st>>>(m, s, p, a);
}

}  // namespace ugkwp
