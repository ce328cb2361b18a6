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

// A failed self-check of a kernel: the error bit, and the first failure's
// check number and value (the access it guards is skipped).
__device__ __forceinline__ void check_failed(const DevState& s, int check, unsigned long long value) {
    atomicCAS(reinterpret_cast<unsigned long long*>(&s.cnt64[CNT_CHECK]), 0ULL,
              ((unsigned long long)check << 48) | (value & 0xffffffffffffULL));
    set_err(s, ERRB_CHECK);
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
__device__ __forceinline__ void sample_scale_body(const DevMesh& m, const DevState& s, const DevParams& p,
                                                  Blk bk) {
    const int nc = m.nc;
    const int cell = bk.id * blockDim.x + threadIdx.x;
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
__global__ void __launch_bounds__(256) k_sample_scale(DevMesh m, DevState s, DevParams p) {
    sample_scale_body<Real>(m, s, p, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// a5 positions: a uniform point in the tet from three uniforms folded cube ->
// prism -> tet (Rocchini & Cignoni, J. Graphics Tools 5(4), 2000).  The
// uniforms are odd multiples of 2^-48 (47 bits of one Philox draw each) and
// the folding runs on their integer numerators, so both precisions start from
// the same exact barycentric weights w_k = N_k 2^-48.
__device__ __forceinline__ void tet_weights(const dm::U4& r, long long N[3]) {
    constexpr long long ONE = 1LL << 48;
    long long a = (long long)(((r.a >> 17) << 1) | 1ULL), b = (long long)(((r.b >> 17) << 1) | 1ULL),
              c = (long long)(((r.c >> 17) << 1) | 1ULL);
    if (a + b > ONE) { a = ONE - a; b = ONE - b; }
    if (b + c > ONE) {
        const long long t = c;
        c = ONE - a - b;
        b = ONE - t;
    } else if (a + b + c > ONE) {
        const long long t = c;
        c = a + b + c - ONE;
        a = ONE - b - t;
    }
    N[0] = a; N[1] = b; N[2] = c;
}

// Error-free sum of two binary32 numbers: s + e = a + b exactly (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Mixed-mode position coordinate: (p0 - A) + ((w1 E1 + w2 E2) + w3 E3) in
// binary32 pairs (high + low, about 44 bits), then rounded to binary32.  f
// points at the coordinate's 8 table entries (stride nc): p0 - A, E1, E2, E3
// as (high, low).  Each product keeps the exact error of its high parts (FMA)
// and the two cross terms; the sums carry their exact errors in the low part.
__device__ __forceinline__ float ff_position(const float* f, int nc, const float wh[3], const float wl[3]) {
    float p[3], e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float eh = f[(size_t)(2 + 2 * k) * nc], el = f[(size_t)(3 + 2 * k) * nc];
        p[k] = wh[k] * eh;
        e[k] = __fmaf_rn(wh[k], eh, -p[k]) + (wh[k] * el + wl[k] * eh);
    }
    float s1, r1;
    two_sum(p[0], p[1], s1, r1);
    float lo = r1 + (e[0] + e[1]);
    float s2, r2;
    two_sum(s1, p[2], s2, r2);
    lo = r2 + (lo + e[2]);
    float s3, r3;
    two_sum(f[0], s2, s3, r3);
    lo = r3 + (lo + f[nc]);
    return s3 + lo;
}

template <class Real>
__device__ __forceinline__ void sample_write_body(const DevMesh& m, const DevState& s, const DevParams& p,
                                                  const PartBufRaw& br, Blk bk) {
    if (s.cnt64[CNT_ERR] & ERRB_CAPACITY) return;
    const PartView<Real> b = view<Real>(br);
    const int nc = m.nc;
    const long long total = s.cnt64[CNT_NSAM];
    const long long step = s.cnt64[CNT_STEP];
    const long long stride = (long long)bk.n * blockDim.x;
    for (long long g = (long long)bk.id * blockDim.x + threadIdx.x; g < total; g += stride) {
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
        if (j >= p.capacity || cell < 0 || cell >= nc) {
            check_failed(s, 9, (unsigned long long)j);
            continue;
        }
        const unsigned long long ida = make_id(step, cell, k - side);
        const unsigned long long id = ida + (unsigned long long)side;
        const bool gp = p.sampling == UGKWP_SAMPLE_GP1;
        long long N[3];
        tet_weights(dm::philox(id, (unsigned long long)step, TAG_SPOS, 0ULL, p.seed, 0ULL), N);
        if constexpr (sizeof(Real) == 4) {
            // mixed mode: velocities in binary32 from U and the spread rounded
            // to binary32; the position offset from the tet's anchor in
            // binary32 pairs, rounded once
            const float4 us = s.usig[cell];
            float X[3];
            if (gp) gp_normals<float>(s.gpc, nc, cell, id, step, p.seed, X);  // every particle on its own
            else pair_normals<float>(ida, step, p.seed, X);
            float wh[3], wl[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                wh[q] = (float)(N[q] >> 24) * 0x1p-24f;
                wl[q] = (float)(N[q] & 0xffffffLL) * 0x1p-48f;
            }
            const float U[3] = {us.x, us.y, us.z};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                b.x[c][j] = ff_position(m.smp_f + (size_t)(8 * c) * nc + cell, nc, wh, wl);
                b.u[c][j] = (gp || side == 0) ? U[c] + us.w * X[c] : U[c] - us.w * X[c];
            }
            if (p.K > 0) b.e[j] = internal_energy<float>(id, step, TAG_SINT, 0ULL, p.K, us.w, p.seed);
        } else {
            const double U[3] = {s.prim[nc + cell], s.prim[2 * nc + cell], s.prim[3 * nc + cell]};
            const double sig =
                p.sampling == UGKWP_SAMPLE_ENERGY_MATCHED ? s.sig[cell] : sqrt(p.R * s.prim[4 * nc + cell]);
            double X[3];
            if (gp) gp_normals<double>(s.gpc, nc, cell, id, step, p.seed, X);
            else pair_normals<double>(ida, step, p.seed, X);
            const double a = (double)N[0] * 0x1p-48, bb = (double)N[1] * 0x1p-48, cc = (double)N[2] * 0x1p-48;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double P0 = m.vtx[(size_t)c * nc + cell];
                const double E1 = m.vtx[(size_t)(3 + c) * nc + cell] - P0;
                const double E2 = m.vtx[(size_t)(6 + c) * nc + cell] - P0;
                const double E3 = m.vtx[(size_t)(9 + c) * nc + cell] - P0;
                b.x[c][j] = P0 + ((a * E1 + bb * E2) + cc * E3);
                b.u[c][j] = (gp || side == 0) ? U[c] + sig * X[c] : U[c] - sig * X[c];
            }
            if (p.K > 0) b.e[j] = internal_energy<double>(id, step, TAG_SINT, 0ULL, p.K, sig, p.seed);
        }
        b.m[j] = s.msam[cell];
        b.cell[j] = cell;
        b.id[j] = id;
    }
}
template <class Real>
__global__ void __launch_bounds__(256) k_sample_write(DevMesh m, DevState s, DevParams p, PartBufRaw br) {
    sample_write_body<Real>(m, s, p, br, Blk{(int)blockIdx.x, (int)gridDim.x});
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
    // the record is one 128-byte line
    __device__ static __forceinline__ void prefetch(const DevMesh& m, int tet) {
        asm volatile("prefetch.global.L1 [%0];" ::"l"(m.trk_f + tet));
    }
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
    // the 144-byte record starts on a 16-byte boundary, so it spans two lines
    __device__ static __forceinline__ void prefetch(const DevMesh& m, int tet) {
        const char* r = reinterpret_cast<const char*>(m.trk_d + tet);
        asm volatile("prefetch.global.L1 [%0];" ::"l"(r));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(r + sizeof(TrkD) - 1));
    }
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

// Thread 0's source of tiles: grabs of TILE_GRAB consecutive tiles from the
// global counter (one atomic per grab), handed out in order, so the tiles a
// block walks increase.  The grab after the current one is reserved when the
// current one starts, so its atomic completes while the current grab's tiles
// are walked (a block stops at its first tile past the end, and every grab it
// still holds then lies past the end too).  Returns the first particle index
// of the next tile.
struct TileQueue {
    long long next = 0, end = 0, ahead = -1;
};

__device__ __forceinline__ long long next_tile(TileQueue& q, int64_t* ctr, int T) {
    if (q.next == q.end) {
        const long long g =
            q.ahead >= 0 ? q.ahead : (long long)atomicAdd(reinterpret_cast<unsigned long long*>(ctr), 1ULL);
        q.next = g * TILE_GRAB;
        q.end = q.next + TILE_GRAB;
        q.ahead = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(ctr), 1ULL);
    }
    return (q.next++) * T;
}

// ---- the walk of one particle, one tet at a time
// Walk state along x0 + u (t - t0): the tet it is in, the face it entered
// through (or last reflected from, skipped in the exit test), its counters.
template <class Real> struct Walk {
    Real x0[3], u[3], t0, t_end;
    int tet, last, ncross, nrefl, nwall, status;
};

// One tet of the face-by-face walk (Sec. 2.2 streaming): the exit face is the
// one with u.n > 0 and the smallest crossing time (d - n.x0)/(u.n), compared
// by cross products (positive denominators) with one division; ties keep the
// lower local face.  Returns true when the walk goes on (into the neighbour,
// or restarted at a wall); false when it ended: stopped inside the tet (xe the
// end point), left the domain (status 2) or passed max_crossings (status 4).
template <class Real, bool KE>
__device__ __forceinline__ bool visit(const DevMesh& m, const DevParams& p, long long step, unsigned long long id,
                                      Walk<Real>& w, Real xe[3], Real& ee) {
    // the tet's neighbour codes, loaded with its planes (they sit in
    // another sector of the tet's record)
    const int4 nbv = Trk<Real>::nbv(m, w.tet);
    int best = -1;
    Real nbest = (Real)0, dbest = (Real)1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k == w.last) continue;
        Real nx, ny, nz, d;
        Trk<Real>::plane(m, w.tet, k, nx, ny, nz, d);
        const Real un = (w.u[0] * nx + w.u[1] * ny) + w.u[2] * nz;
        if (un > (Real)0) {
            const Real xn = (w.x0[0] * nx + w.x0[1] * ny) + w.x0[2] * nz;
            const Real num = d - xn;
            if (best < 0 || num * dbest < nbest * un) { best = k; nbest = num; dbest = un; }
        }
    }
    Real sbest = best >= 0 ? nbest / dbest : (Real)0;
    const Real rem = w.t_end - w.t0;
    if (best < 0 || sbest >= rem) {
#pragma unroll
        for (int c = 0; c < 3; ++c) xe[c] = w.x0[c] + w.u[c] * rem;
        return false;
    }
    if (sbest < (Real)0) sbest = (Real)0;
    ++w.ncross;
    if (w.ncross > p.max_crossings) {
        w.status |= 4;
#pragma unroll
        for (int c = 0; c < 3; ++c) xe[c] = w.x0[c];
        return false;
    }
    const int code = best == 0 ? nbv.x : best == 1 ? nbv.y : best == 2 ? nbv.z : nbv.w;
    if (code >= 0) {
        const int nt = code >> 2;
        if constexpr (sizeof(Real) == 4) {
            // mixed mode: the segment start moves into the next tet's frame
            // (the anchors' difference, exact in binary32, sits in the
            // record's line loaded for the planes)
            const float* da = m.trk_f[w.tet].da + 3 * best;
            w.x0[0] = w.x0[0] + da[0];
            w.x0[1] = w.x0[1] + da[1];
            w.x0[2] = w.x0[2] + da[2];
        }
        w.tet = nt;
        w.last = code & 3;
        return true;
    }
    const int bi = -1 - code;
    const DevBc& bc = p.bc[m.bf_tag[bi]];
    if (bc.type == UGKWP_BC_FARFIELD || bc.type == UGKWP_BC_OUTFLOW) {
        w.status |= 2;
        return false;
    }
    Real xh[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) xh[c] = w.x0[c] + w.u[c] * sbest;
    if (bc.type == UGKWP_BC_SPECULAR) {
        Real nx, ny, nz, d;
        Trk<Real>::plane(m, w.tet, best, nx, ny, nz, d);
        const Real un = (w.u[0] * nx + w.u[1] * ny) + w.u[2] * nz;
        const Real two = un + un;
        w.u[0] = w.u[0] - two * nx;
        w.u[1] = w.u[1] - two * ny;
        w.u[2] = w.u[2] - two * nz;
    } else {
        // diffuse re-emission, full accommodation: |u_n| = sqrt(-2 R T_w ln eta),
        // tangential components U_w,t + sqrt(R T_w) N(0,1)
        const dm::U4 r = dm::philox(id, (unsigned long long)step, TAG_WALL, (unsigned long long)w.nwall, p.seed, 0ULL);
        if constexpr (sizeof(Real) == 4) {
            // mixed mode: binary32 from the wall constants and the face frame
            // rounded to binary32
            const float vn = sqrtf(bc.c2rt_f * dm::f_log(dm::u01f(r.a)));
            const float rad = sqrtf(-2.0f * dm::f_log(dm::u01f(r.b)));
            float sn, cs;
            dm::f_sincos2pi(dm::u01f(r.c), &sn, &cs);
            const int nbf = m.nbf;
            const float v1 = m.bf_f[(size_t)9 * nbf + bi] + bc.sw_f * (rad * cs);
            const float v2 = m.bf_f[(size_t)10 * nbf + bi] + bc.sw_f * (rad * sn);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                w.u[c] = ((-vn) * m.bf_f[(size_t)c * nbf + bi] + v1 * m.bf_f[(size_t)(3 + c) * nbf + bi]) +
                         v2 * m.bf_f[(size_t)(6 + c) * nbf + bi];
            if constexpr (KE)
                ee = internal_energy<float>(id, step, TAG_WINT, 2ULL * (unsigned long long)w.nwall, p.K, bc.sw_f, p.seed);
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
            for (int c = 0; c < 3; ++c) w.u[c] = (Real)(((-vn) * n3[c] + v1 * t1[c]) + v2 * t2[c]);
            if constexpr (KE)
                ee = (Real)internal_energy<double>(id, step, TAG_WINT, 2ULL * (unsigned long long)w.nwall, p.K, sw, p.seed);
        }
        ++w.nwall;
    }
    ++w.nrefl;
#pragma unroll
    for (int c = 0; c < 3; ++c) w.x0[c] = xh[c];
    w.t0 = w.t0 + sbest;
    w.last = best;
    return true;
}

// A particle whose walk ended, ready for the outputs.
template <class Real> struct Ended {
    bool active, survivor, mover, exited;
    int tet, c0;
    Real xe[3], ue[3], us[3], es, ee;
    double mm;
    unsigned long long id;
};

// Walks that did not end in their first tet wait in shared memory (structure
// of arrays, QCAP entries per block) until a tile's worth of them has
// gathered; the block then walks one tile's worth on in full warps.  Before a
// tile's pushes fewer than T walks wait, so 2T entries always suffice.  An entry holds the walk state,
// the particle's internal energy (KE) and its slot in the buffer, from which
// the rest of the particle is read again when the walk ends.
template <class Real, bool KE, int T> struct WalkQueue {
    static constexpr int QCAP = 2 * T;
    Real x0[3][QCAP], u[3][QCAP], t0[QCAP], t_end[QCAP], ee[KE ? QCAP : 1];
    int tet[QCAP], last[QCAP], ncross[QCAP], nrefl[QCAP], nwall[QCAP], flags[QCAP];  // flags: status | coll << 3
    long long slot[QCAP];
    int count;
};

// KE: the particles carry an internal energy (K > 0).  THREADS: particles per
// tile (one per thread).
template <class Real, bool KE, int THREADS>
__device__ __forceinline__ void track_body(const DevMesh& m, const DevState& s, const DevParams& p,
                                           const PartBufRaw& br, const PartBufRaw& nr, const PartBufRaw& ar) {
    constexpr int NW = THREADS / 32;
    using Q = WalkQueue<Real, KE, THREADS>;
    // (block-uniform: another block may set the bit while this one starts)
    if (__syncthreads_or(threadIdx.x == 0 && (s.cnt64[CNT_ERR] & ERRB_CAPACITY))) return;
    const PartView<Real> b = view<Real>(br);   // this step's particles, sorted by cell (holes: cell -1)
    const PartView<Real> nxt = view<Real>(nr);  // the next step's survivors, in their end cells' buckets
    const PartView<Real> mv = view<Real>(ar);  // mover list: x = u at start, u = u at end
    const long long n = s.cnt64[CNT_N_B];
    const long long step = s.cnt64[CNT_STEP];
    const double dt = s.dt[0];
    const Real dtR = (Real)dt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // slot bookkeeping in two sets, alternating between output rounds, so
    // that no barrier is needed after a round's stores: a set is rewritten
    // two rounds later, after two barriers every warp has passed
    __shared__ int sh_cnt[2][NW];
    __shared__ long long sh_base[2], sh_tile[2];
    __shared__ int sh_qc;  // queue size after the last output round
    const long long wtot = s.cnt64[CNT_WTOT];  // overflow slots start after the buckets
    int par = 0;
    __shared__ unsigned long long sh_red[NW][8];
    __shared__ Q q;
    // per-thread counters, reduced once per block at the end
    unsigned c_valid = 0, c_coll = 0, c_exit = 0, c_lost = 0, c_cross = 0, c_wall = 0, c_surv = 0;
    // tiles of THREADS particles are taken from a global counter, so that
    // blocks that start late (or walk short paths) take fewer tiles
    TileQueue tq;  // thread 0's
    if (threadIdx.x == 0) {
        q.count = 0;
        sh_qc = 0;
        sh_tile[0] = next_tile(tq, &s.cnt64[CNT_TILE], THREADS);
    }
    __syncthreads();

    // ---- outputs of the particles whose walks ended this round (one per
    // lane or none): the survivor's slot in its end cell's bucket, the
    // survivors' mass per end cell, the counters, the mover record.  Contains
    // the block's two barriers of the round; with `advance`, thread 0 also
    // takes the next tile.
    auto emit = [&](const Ended<Real>& e, bool advance, int qtake) {
        // a11: each survivor goes to the bucket of its end cell in the next
        // buffer, so the next step finds the particles sorted by cell.  Lanes
        // with the same end cell take consecutive slots from the cell's count
        // (one atomic per group); the count is also the cell's survivor count
        // N_left of the next step.  A survivor beyond its bucket takes an
        // overflow slot after the buckets.  The group's first slot is read
        // after the round's barriers, so the atomic's round trip overlaps them.
        const int key = e.survivor ? e.tet : -1;
        const unsigned peers = __match_any_sync(FULL, key);
        const int leader = __ffs(peers) - 1;
        int sfirst = 0;
        if (lane == leader && key >= 0) sfirst = atomicAdd(&s.nleft_next[key], __popc(peers));
        // survivors' fixed-point mass per end cell: segmented reduction over
        // lanes with equal keys in a row, one atomic per run
        {
            long long v = 0;
            if (e.survivor && !fixed_of_mass(e.mm, p.exps[0], v)) set_err(s, ERRB_FIXED_OVERFLOW);
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
        c_surv += e.survivor ? 1u : 0u;
        // movers: one slot reservation per block and round
        const unsigned mmask = __ballot_sync(FULL, e.mover);
        if (lane == 0) sh_cnt[par][warp] = __popc(mmask);
        __syncthreads();
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
            // the walks taken from the queue this round leave it (every
            // thread read its entry before the barrier above)
            q.count -= qtake;
            // the queue's size as every warp must see it after this round: a
            // warp that leaves the round early may already push the next
            // tile's walks into q.count before a slower warp reads it
            sh_qc = q.count;
            // the next tile, in the other set (its last readers read it before
            // the barrier above); a round without a new tile keeps the current one
            sh_tile[par ^ 1] = advance ? next_tile(tq, &s.cnt64[CNT_TILE], THREADS) : sh_tile[par];
        }
        __syncthreads();
        const int srank = __shfl_sync(FULL, sfirst, leader) + __popc(peers & ((1u << lane) - 1u));
        if (e.survivor) {
            long long j = -1;
            if (srank < s.wcap[e.tet]) {
                j = (long long)s.woff[e.tet] + srank;
            } else {
                const long long o = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&s.cnt64[CNT_OVF]), 1ULL);
                if (o < p.capacity - wtot) j = wtot + o;
                else set_err(s, ERRB_CAPACITY);
            }
            if (j >= p.capacity) {
                check_failed(s, 6, (unsigned long long)j);
                j = -1;
            }
            if (j >= 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    nxt.x[c][j] = e.xe[c];
                    nxt.u[c][j] = e.ue[c];
                }
                nxt.m[j] = e.mm;
                nxt.cell[j] = e.tet;
                nxt.id[j] = e.id;
                if constexpr (KE) nxt.e[j] = e.ee;
            }
        }
        const long long mj = sh_base[par] + sh_cnt[par][warp] + __popc(mmask & ((1u << lane) - 1u));
        if (e.mover && mj >= p.capacity) check_failed(s, 7, (unsigned long long)mj);
        if (e.mover && mj < p.capacity) {
            const long long j = mj;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                mv.x[c][j] = e.us[c];
                mv.u[c][j] = e.ue[c];
            }
            mv.m[j] = e.mm;
            mv.cell[j] = e.c0;
            mv.id[j] = ((unsigned long long)(unsigned)e.tet << 1) | (e.exited ? 1ULL : 0ULL);
            if constexpr (KE) {
                mv.e[j] = e.es;
                mv.e2[j] = e.ee;
            }
        }
        par ^= 1;
    };

    // The end of a walk: removal (a9), counters, the mover flag (a8: a
    // particle that ends in its start cell with its velocity unchanged
    // contributes nothing to the counting flux; the others are listed for the
    // binary64 flux pass).
    auto finish = [&](const Walk<Real>& w, bool coll, Ended<Real>& e) {
        e.active = true;
        e.exited = w.status & 2;
        const bool lost = w.status & 4;
        e.survivor = !e.exited && (!coll || lost);
        const int status = w.status | ((coll && !lost && !e.exited) ? 1 : 0);
        e.tet = w.tet;
        e.mover = e.exited || w.tet != e.c0 || w.nrefl > 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) e.ue[c] = w.u[c];
        c_coll += status & 1;
        c_exit += (status >> 1) & 1;
        c_lost += (status >> 2) & 1;
        c_cross += w.ncross;
        c_wall += w.nwall;
    };

    for (;;) {
        const long long bb = sh_tile[par];  // block-uniform
        const bool have_tile = bb < n;
        if (!have_tile && sh_qc == 0) break;
        // ---- a new tile: load, t_f, the first tet of every walk
        Ended<Real> e;
        e.active = e.survivor = e.mover = e.exited = false;
        e.tet = e.c0 = -1;
        e.es = e.ee = (Real)0;
        e.mm = 0.0;
        e.id = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) e.xe[c] = e.ue[c] = e.us[c] = (Real)0;
        if (have_tile) {
            const long long i = bb + threadIdx.x;
            // the whole slot is read at once (one round trip; the arrays hold
            // whole tiles, so slots past n are inside them and ignored); the
            // slot's start cell -1 marks a hole of a survivor bucket
            Walk<Real> w;
            const int cell_i = b.cell[i];
            const unsigned long long id_i = b.id[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                w.x0[c] = b.x[c][i];
                w.u[c] = b.u[c][i];
            }
            const double m_i = b.m[i];
            Real e_i = (Real)0;
            if constexpr (KE) e_i = b.e[i];
            const int c0 = i < n ? cell_i : -1;
            if (c0 >= 0) {
                // the start tet's record is on its way to L1 during the t_f draw
                Trk<Real>::prefetch(m, c0);
                e.id = id_i;
                e.mm = m_i;
                e.es = e_i;
                e.ee = e.es;
                e.c0 = c0;
#pragma unroll
                for (int c = 0; c < 3; ++c) e.us[c] = w.u[c];
                c_valid += 1;
                // a6: t_f = min(-tau ln eta, dt) for the particles left from the last step
                w.t_end = dtR;
                bool coll = false;
                if ((long long)(e.id >> 40) != step) {
                    // Philox4x32-10, counter (id low, id high, step, TAG_TF), key (seed low, seed high)
                    const unsigned long long r = dm::philox32_2((unsigned)e.id, (unsigned)(e.id >> 32), (unsigned)step,
                                                                (unsigned)TAG_TF, (unsigned)p.seed,
                                                                (unsigned)(p.seed >> 32));
                    const Real tf = Trk<Real>::tf(Trk<Real>::tau(s, c0), r);
                    if (tf < dtR) { coll = true; w.t_end = tf; }
                }
                // a7: the walk's first tet
                w.t0 = (Real)0;
                w.tet = c0;
                w.last = -1;
                w.ncross = w.nrefl = w.nwall = w.status = 0;
                if (visit<Real, KE>(m, p, step, e.id, w, e.xe, e.ee)) {
                    // the walk goes on: it waits in the queue
                    const int k = atomicAdd(&q.count, 1);
                    if (k >= Q::QCAP) check_failed(s, 5, (unsigned long long)k);
                    else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        q.x0[c][k] = w.x0[c];
                        q.u[c][k] = w.u[c];
                    }
                    q.t0[k] = w.t0;
                    q.t_end[k] = w.t_end;
                    if constexpr (KE) q.ee[k] = e.ee;
                    q.tet[k] = w.tet;
                    q.last[k] = w.last;
                    q.ncross[k] = w.ncross;
                    q.nrefl[k] = w.nrefl;
                    q.nwall[k] = w.nwall;
                    q.flags[k] = w.status | (coll ? 8 : 0);
                    q.slot[k] = i;
                    }
                } else {
                    finish(w, coll, e);
                }
            }
        }
        emit(e, have_tile, 0);
        // ---- the queued walks, in full warps once a tile's worth of them has
        // gathered (or once the tiles are done)
        const int qc = sh_qc;  // block-uniform: set between the round's barriers
        if (qc >= THREADS || (!have_tile && qc > 0)) {
            const int take = qc < THREADS ? qc : THREADS;
            Ended<Real> f;
            f.active = f.survivor = f.mover = f.exited = false;
            f.tet = f.c0 = -1;
            f.es = f.ee = (Real)0;
            f.mm = 0.0;
            f.id = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) f.xe[c] = f.ue[c] = f.us[c] = (Real)0;
            if ((int)threadIdx.x < take) {
                const int k = qc - take + threadIdx.x;
                Walk<Real> w;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    w.x0[c] = q.x0[c][k];
                    w.u[c] = q.u[c][k];
                }
                w.t0 = q.t0[k];
                w.t_end = q.t_end[k];
                w.tet = q.tet[k];
                w.last = q.last[k];
                w.ncross = q.ncross[k];
                w.nrefl = q.nrefl[k];
                w.nwall = q.nwall[k];
                const int fl = q.flags[k];
                w.status = fl & 7;
                const bool coll = fl & 8;
                const long long i = q.slot[k];
                // the rest of the particle, read again from its slot
                f.id = b.id[i];
                f.c0 = b.cell[i];
                f.mm = b.m[i];
#pragma unroll
                for (int c = 0; c < 3; ++c) f.us[c] = b.u[c][i];
                if constexpr (KE) {
                    f.es = b.e[i];
                    f.ee = q.ee[k];
                }
                while (visit<Real, KE>(m, p, step, f.id, w, f.xe, f.ee)) {
                }
                finish(w, coll, f);
            }
            emit(f, false, take);
        }
    }
    // ---- counters: one atomic per block and counter
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
template <class Real, bool KE, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_track(DevMesh m, DevState s, DevParams p, PartBufRaw br,
                                                                  PartBufRaw nr, PartBufRaw ar) {
    track_body<Real, KE, THREADS>(m, s, p, br, nr, ar);
}

// Same bits (a particle's velocity and internal energy are unchanged unless it
// met a wall).
__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
__device__ __forceinline__ bool same_bits(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b);
}

// Counting flux of the listed movers: -phi(u_start) at the start cell and, unless
// the particle left the domain, +phi(u_end) at the end cell (full warps of
// binary64 work, kept out of the tracking kernel).  phi(u_end) is phi(u_start)
// for the movers that met no wall.

template <class Real>
__device__ __forceinline__ void movers_body(const DevMesh& m, const DevState& s, const DevParams& p,
                                            const PartBufRaw& ar, Blk bk) {
    if (__syncthreads_or(threadIdx.x == 0 && (s.cnt64[CNT_ERR] & ERRB_CAPACITY))) return;
    const PartView<Real> mv = view<Real>(ar);
    const long long n = s.cnt64[CNT_RESV];
    const int nc = m.nc;
    const int lane = threadIdx.x & 31;
    unsigned long long* pf = reinterpret_cast<unsigned long long*>(s.pflux);
    // movers whose end velocity differs from their start velocity (they met
    // a wall): their end phi is taken after the block's pass, packed into
    // whole warps, since binary64 work costs a warp its full issue time
    __shared__ int wall_j[256];
    __shared__ int n_wall;
    for (long long base = (long long)bk.id * 256; base < n; base += (long long)bk.n * 256) {
        if (threadIdx.x == 0) n_wall = 0;
        __syncthreads();
        const long long j = base + threadIdx.x;
        const bool valid = j < n;
        Real us[3] = {(Real)0, (Real)0, (Real)0};
        double mm = 0.0;
        int c0 = -1, c1 = -1;
        bool exited = true;
        long long q0[5] = {0, 0, 0, 0, 0};
        if (valid) {
            Real ue[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) { us[c] = mv.x[c][j]; ue[c] = mv.u[c][j]; }
            mm = mv.m[j];
            c0 = mv.cell[j];
            const unsigned long long code = mv.id[j];
            c1 = (int)(code >> 1);
            exited = code & 1ULL;
            // a record outside the mesh is reported and skipped
            if (c0 < 0 || c0 >= nc || (!exited && (c1 < 0 || c1 >= nc))) {
                check_failed(s, 8, (unsigned long long)j);
                c0 = -1;
                exited = true;
            }
            const Real es = mv.e ? mv.e[j] : (Real)0, ee = mv.e2 ? mv.e2[j] : (Real)0;
            if (!phi_q(us, es, mm, p, q0)) set_err(s, ERRB_FIXED_OVERFLOW);
            const bool same = same_bits(us[0], ue[0]) && same_bits(us[1], ue[1]) && same_bits(us[2], ue[2]) &&
                              same_bits(es, ee);
            if (!exited && !same) wall_j[atomicAdd(&n_wall, 1)] = threadIdx.x;
            if (!exited && same) {
                // +phi at the end cell: the start's phi
#pragma unroll
                for (int q = 0; q < 5; ++q) atomicAdd(&pf[(size_t)q * nc + c1], (unsigned long long)q0[q]);
            }
        }
        // -phi at the start cell, summed over runs of equal start cells within
        // the warp (the list is ordered by start cell within each tracking
        // tile), one atomic per run and quantity
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
            if (tail && c0 >= 0) atomicAdd(&pf[(size_t)q * nc + c0], (unsigned long long)v);
        }
        __syncthreads();
        // the block's wall movers: +phi(u_end) at the end cell
        for (int t = threadIdx.x; t < n_wall; t += 256) {
            const long long jw = base + wall_j[t];
            Real ue[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) ue[c] = mv.u[c][jw];
            const Real ee = mv.e2 ? mv.e2[jw] : (Real)0;
            long long q1[5];
            if (!phi_q(ue, ee, mv.m[jw], p, q1)) set_err(s, ERRB_FIXED_OVERFLOW);
            const int cw = (int)(mv.id[jw] >> 1);
#pragma unroll
            for (int q = 0; q < 5; ++q) atomicAdd(&pf[(size_t)q * nc + cw], (unsigned long long)q1[q]);
        }
        __syncthreads();
    }
}
template <class Real>
__global__ void __launch_bounds__(256) k_movers(DevMesh m, DevState s, DevParams p, PartBufRaw ar) {
    movers_body<Real>(m, s, p, ar, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// ---- fused batches
__device__ __forceinline__ int member_of(const int32_t* off, int n) {
    int lo = 0, hi = n;  // off[lo] <= blockIdx.x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid;
    }
    return lo;
}
template <class Real>
__global__ void __launch_bounds__(256) k_sample_scale_b(const __grid_constant__ BatchChunk c) {
    const int32_t* off = c.off[BCL_CELLS];
    const int i = member_of(off, c.n);
    sample_scale_body<Real>(c.mem[i].m, c.mem[i].s, c.mem[i].p, Blk{(int)blockIdx.x - off[i], off[i + 1] - off[i]});
}
// The particle kernels take every member of the chunk in turn on the whole grid.
template <class Real>
__global__ void __launch_bounds__(256) k_sample_write_b(const __grid_constant__ BatchChunk c) {
    for (int k = 0; k < c.n; ++k)
        sample_write_body<Real>(c.mem[k].m, c.mem[k].s, c.mem[k].p, c.mem[k].a, Blk{(int)blockIdx.x, (int)gridDim.x});
}
// Tiles come from each member's own counter; a block starts at member
// blockIdx.x mod n, so that the blocks spread over the members' counters.
template <class Real, bool KE, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_track_b(const __grid_constant__ BatchChunk c) {
    for (int k = 0; k < c.n; ++k) {
        const BatchMember& e = c.mem[((int)blockIdx.x + k) % c.n];
        track_body<Real, KE, THREADS>(e.m, e.s, e.p, e.a, e.b, e.mv);
        __syncthreads();
    }
}
template <class Real>
__global__ void __launch_bounds__(256) k_movers_b(const __grid_constant__ BatchChunk c) {
    for (int k = 0; k < c.n; ++k)
        movers_body<Real>(c.mem[k].m, c.mem[k].s, c.mem[k].p, c.mem[k].mv, Blk{(int)blockIdx.x, (int)gridDim.x});
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
template <class Real, bool KE>
void track_shape(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& b, const PartBufRaw& nxt,
                 const PartBufRaw& movers, const TrackShape& sh, int blocks, cudaStream_t st) {
    if (sh.threads == 256) k_track<Real, KE, 256><<<blocks, 256, 0, st>>>(m, s, p, b, nxt, movers);
    else k_track<Real, KE, 128><<<blocks, 128, 0, st>>>(m, s, p, b, nxt, movers);
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
// The preferred carveout of the particle kernels of one particle type.
template <class Real, bool KE> cudaError_t configure_type(int carveout) {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    };
    set(k_track<Real, KE, 128>);
    set(k_track<Real, KE, 256>);
    set(k_sample_write<Real>);
    set(k_sample_scale<Real>);
    set(k_movers<Real>);
    set(k_track_b<Real, KE, 128>);
    set(k_track_b<Real, KE, 256>);
    set(k_sample_write_b<Real>);
    set(k_sample_scale_b<Real>);
    set(k_movers_b<Real>);
    return e;
}
}  // namespace

cudaError_t configure_particle_kernels(const DevParams& p, int carveout) {
    if (p.precision == UGKWP_MIXED) return p.K > 0 ? configure_type<float, true>(carveout) : configure_type<float, false>(carveout);
    return p.K > 0 ? configure_type<double, true>(carveout) : configure_type<double, false>(carveout);
}

void launch_movers(const DevMesh& m, const DevState& s, const DevParams& p, const PartBufRaw& a, int blocks, cudaStream_t st) {
    if (p.precision == UGKWP_MIXED) k_movers<float><<<blocks, 256, 0, st>>>(m, s, p, a);
    else k_movers<double><<<blocks, 256, 0, st>>>(m, s, p, a);
}

void launch_sample_scale_batch(const BatchChunk& c, int blocks, int precision, cudaStream_t st) {
    if (precision == UGKWP_MIXED) k_sample_scale_b<float><<<blocks, 256, 0, st>>>(c);
    else k_sample_scale_b<double><<<blocks, 256, 0, st>>>(c);
}
void launch_sample_write_batch(const BatchChunk& c, int blocks, int precision, cudaStream_t st) {
    if (precision == UGKWP_MIXED) k_sample_write_b<float><<<blocks, 256, 0, st>>>(c);
    else k_sample_write_b<double><<<blocks, 256, 0, st>>>(c);
}
namespace {
template <class Real, bool KE>
void track_batch_shape(const BatchChunk& c, const TrackShape& sh, int blocks, cudaStream_t st) {
    if (sh.threads == 256) k_track_b<Real, KE, 256><<<blocks, 256, 0, st>>>(c);
    else k_track_b<Real, KE, 128><<<blocks, 128, 0, st>>>(c);
}
}  // namespace
void launch_track_batch(const BatchChunk& c, int precision, bool ke, const TrackShape& sh, int blocks,
                        cudaStream_t st) {
    if (precision == UGKWP_MIXED) {
        if (ke) track_batch_shape<float, true>(c, sh, blocks, st);
        else track_batch_shape<float, false>(c, sh, blocks, st);
    } else {
        if (ke) track_batch_shape<double, true>(c, sh, blocks, st);
        else track_batch_shape<double, false>(c, sh, blocks, st);
    }
}
void launch_movers_batch(const BatchChunk& c, int blocks, int precision, cudaStream_t st) {
    if (precision == UGKWP_MIXED) k_movers_b<float><<<blocks, 256, 0, st>>>(c);
    else k_movers_b<double><<<blocks, 256, 0, st>>>(c);
}

}  // namespace ugkwp
