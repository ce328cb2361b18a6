// Device elementary functions and counter-based random numbers for the
// particle path.  They are evaluated with IEEE +, -, *, / and sqrt only and the
// translation units that include this header are compiled with --fmad=false,
// so each value is reproducible bit for bit on any IEEE-754 machine that
// evaluates the same operation sequence.  The methods:
//
//   d_exp       Cody-Waite reduction x = k ln2 + r (ln2 = 32-bit head + tail),
//               Horner evaluation of the degree-13 Taylor polynomial of e^r,
//               exact scaling by 2^k (two steps below the normal range).
//   d_log       x = 2^e m, m in (sqrt(1/2), sqrt(2)], f = (m-1)/(m+1),
//               log m = 2f (1 + s/3 + ... + s^11/23), s = f^2.
//   f_log       the same identity in binary32, series to s^5/11.
//   d_sincos2pi sin/cos of 2 pi u by exact quarter-turn reduction and the
//               Taylor series of sin and cos on [-pi/4, pi/4]; f_sincos2pi the
//               same in binary32 (sin to th^11/11!, cos to th^12/12!).
//   philox      Philox4x64-10 and (philox32_2) Philox4x32-10 of Salmon et al. (SC'11).
#pragma once
#include <cstdint>

namespace ugkwp {
namespace dm {

__device__ __forceinline__ double pow2i(int k) {
    return __longlong_as_double((long long)(k + 1023) << 52);
}

// Taylor coefficients 1/j!, j = 0..20, as exact-rounded binary64.
__device__ __forceinline__ double inv_fact(int j) {
    switch (j) {
        case 0: return 1.0;
        case 1: return 1.0;
        case 2: return 0x1.0000000000000p-1;
        case 3: return 0x1.5555555555555p-3;
        case 4: return 0x1.5555555555555p-5;
        case 5: return 0x1.1111111111111p-7;
        case 6: return 0x1.6c16c16c16c17p-10;
        case 7: return 0x1.a01a01a01a01ap-13;
        case 8: return 0x1.a01a01a01a01ap-16;
        case 9: return 0x1.71de3a556c734p-19;
        case 10: return 0x1.27e4fb7789f5cp-22;
        case 11: return 0x1.ae64567f544e4p-26;
        case 12: return 0x1.1eed8eff8d898p-29;
        case 13: return 0x1.6124613a86d09p-33;
        case 14: return 0x1.93974a8c07c9dp-37;
        case 15: return 0x1.ae7f3e733b81fp-41;
        case 16: return 0x1.ae7f3e733b81fp-45;
        case 17: return 0x1.952c77030ad4ap-49;
        case 18: return 0x1.6827863b97d97p-53;
        case 19: return 0x1.2f49b46814157p-57;
        default: return 0x1.e542ba4020225p-62;
    }
}

// 1/(2j+1), j = 1..11, binary64.
__device__ __forceinline__ double inv_odd(int j) {
    switch (j) {
        case 1: return 0x1.5555555555555p-2;
        case 2: return 0x1.999999999999ap-3;
        case 3: return 0x1.2492492492492p-3;
        case 4: return 0x1.c71c71c71c71cp-4;
        case 5: return 0x1.745d1745d1746p-4;
        case 6: return 0x1.3b13b13b13b14p-4;
        case 7: return 0x1.1111111111111p-4;
        case 8: return 0x1.e1e1e1e1e1e1ep-5;
        case 9: return 0x1.af286bca1af28p-5;
        case 10: return 0x1.8618618618618p-5;
        default: return 0x1.642c8590b2164p-5;
    }
}

__device__ __forceinline__ double d_exp(double x) {
    if (x != x) return x;
    if (x > 709.782712893384) return __longlong_as_double(0x7ff0000000000000LL);
    if (x < -745.2) return 0.0;
    const double k = floor(x * 0x1.71547652b82fep+0 + 0.5);
    const double r = (x - k * 0x1.62e42fee00000p-1) - k * 0x1.a39ef35793c76p-33;
    double p = inv_fact(13);
#pragma unroll
    for (int j = 12; j >= 0; --j) p = p * r + inv_fact(j);
    const int ki = (int)k;
    if (ki > 1023) return (p * pow2i(ki - 1)) * 2.0;
    if (ki >= -1022) return p * pow2i(ki);
    return (p * pow2i(ki + 60)) * pow2i(-60);
}

__device__ __forceinline__ double d_log(double x) {
    if (x != x || x < 0.0) return __longlong_as_double(0x7ff8000000000000LL);
    if (x == 0.0) return __longlong_as_double((long long)0xfff0000000000000ULL);
    if (x == __longlong_as_double(0x7ff0000000000000LL)) return x;
    int e_adj = 0;
    if (x < 0x1p-1022) { x = x * 0x1p54; e_adj = -54; }
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = __longlong_as_double((long long)((b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL));
    if (m > 0x1.6a09e667f3bcdp+0) { m = m * 0.5; e += 1; }
    e += e_adj;
    const double f = (m - 1.0) / (m + 1.0);
    const double s = f * f;
    double q = inv_odd(11);
#pragma unroll
    for (int j = 10; j >= 1; --j) q = q * s + inv_odd(j);
    const double f2 = f + f;
    const double logm = f2 + (f2 * s) * q;
    const double de = (double)e;
    return de * 0x1.62e42fee00000p-1 + (de * 0x1.a39ef35793c76p-33 + logm);
}

__device__ __forceinline__ float f_log(float x) {
    if (x != x || x < 0.0f) return __int_as_float(0x7fc00000);
    if (x == 0.0f) return __int_as_float((int)0xff800000u);
    if (x == __int_as_float(0x7f800000)) return x;
    int e_adj = 0;
    if (x < 0x1p-126f) { x = x * 0x1p24f; e_adj = -24; }
    const unsigned b = (unsigned)__float_as_int(x);
    int e = (int)((b >> 23) & 0xff) - 127;
    float m = __int_as_float((int)((b & 0x007fffffu) | 0x3f800000u));
    if (m > 0x1.6a09e6p+0f) { m = m * 0.5f; e += 1; }
    e += e_adj;
    const float f = (m - 1.0f) / (m + 1.0f);
    const float s = f * f;
    float q = 0x1.745d18p-4f;                 // 1/11
    q = q * s + 0x1.c71c72p-4f;               // 1/9
    q = q * s + 0x1.24924ap-3f;               // 1/7
    q = q * s + 0x1.99999ap-3f;               // 1/5
    q = q * s + 0x1.555556p-2f;               // 1/3
    const float f2 = f + f;
    const float logm = f2 + (f2 * s) * q;
    const float de = (float)e;
    return de * 0x1.62e4p-1f + (de * 0x1.7f7d1cp-20f + logm);
}

__device__ __forceinline__ void d_sincos2pi(double u, double* sn_out, double* cs_out) {
    const double q = 4.0 * u;
    const double j = floor(q + 0.5);
    const double th = (q - j) * 0x1.921fb54442d18p+0;
    const double t2 = th * th;
    // sin: odd coefficients (-1)^k / (2k+1)!, k = 9 .. 1
    double ps = -inv_fact(19);
    ps = ps * t2 + inv_fact(17);
    ps = ps * t2 - inv_fact(15);
    ps = ps * t2 + inv_fact(13);
    ps = ps * t2 - inv_fact(11);
    ps = ps * t2 + inv_fact(9);
    ps = ps * t2 - inv_fact(7);
    ps = ps * t2 + inv_fact(5);
    ps = ps * t2 - inv_fact(3);
    const double sn = th + (th * t2) * ps;
    // cos: even coefficients (-1)^k / (2k)!, k = 10 .. 1
    double pc = inv_fact(20);
    pc = pc * t2 - inv_fact(18);
    pc = pc * t2 + inv_fact(16);
    pc = pc * t2 - inv_fact(14);
    pc = pc * t2 + inv_fact(12);
    pc = pc * t2 - inv_fact(10);
    pc = pc * t2 + inv_fact(8);
    pc = pc * t2 - inv_fact(6);
    pc = pc * t2 + inv_fact(4);
    pc = pc * t2 - inv_fact(2);
    const double cs = 1.0 + t2 * pc;
    const int quadrant = ((int)j) & 3;
    if (quadrant == 0) { *sn_out = sn; *cs_out = cs; }
    else if (quadrant == 1) { *sn_out = cs; *cs_out = -sn; }
    else if (quadrant == 2) { *sn_out = -sn; *cs_out = -cs; }
    else { *sn_out = -cs; *cs_out = sn; }
}

// Binary32 variant (mixed-mode particles): 4u and q - j are exact for u on
// the 2^-24 grid of u01f.
__device__ __forceinline__ void f_sincos2pi(float u, float* sn_out, float* cs_out) {
    const float q = 4.0f * u;
    const float j = floorf(q + 0.5f);
    const float th = (q - j) * 0x1.921fb6p+0f;
    const float t2 = th * th;
    float ps = -0x1.ae6456p-26f;   // -1/11!
    ps = ps * t2 + 0x1.71de3ap-19f;  // +1/9!
    ps = ps * t2 - 0x1.a01a02p-13f;  // -1/7!
    ps = ps * t2 + 0x1.111112p-7f;   // +1/5!
    ps = ps * t2 - 0x1.555556p-3f;   // -1/3!
    const float sn = th + (th * t2) * ps;
    float pc = 0x1.1eed8ep-29f;    // +1/12!
    pc = pc * t2 - 0x1.27e4fcp-22f;  // -1/10!
    pc = pc * t2 + 0x1.a01a02p-16f;  // +1/8!
    pc = pc * t2 - 0x1.6c16c2p-10f;  // -1/6!
    pc = pc * t2 + 0x1.555556p-5f;   // +1/4!
    pc = pc * t2 - 0x1p-1f;          // -1/2!
    const float cs = 1.0f + t2 * pc;
    const int quadrant = ((int)j) & 3;
    if (quadrant == 0) { *sn_out = sn; *cs_out = cs; }
    else if (quadrant == 1) { *sn_out = cs; *cs_out = -sn; }
    else if (quadrant == 2) { *sn_out = -sn; *cs_out = -cs; }
    else { *sn_out = -cs; *cs_out = sn; }
}

struct U4 { unsigned long long a, b, c, d; };

__device__ __forceinline__ U4 philox(unsigned long long c0, unsigned long long c1, unsigned long long c2,
                                     unsigned long long c3, unsigned long long k0, unsigned long long k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long hi0 = __umul64hi(0xD2E7470EE14C6C93ULL, c0);
        const unsigned long long lo0 = 0xD2E7470EE14C6C93ULL * c0;
        const unsigned long long hi1 = __umul64hi(0xCA5A826395121157ULL, c2);
        const unsigned long long lo1 = 0xCA5A826395121157ULL * c2;
        const unsigned long long n0 = hi1 ^ c1 ^ k0;
        const unsigned long long n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    return U4{c0, c1, c2, c3};
}

// Philox4x32-10 (same paper, 32x32->64 multiplies); returns output words 0
// and 1 as one 64-bit value (word 0 high).
__device__ __forceinline__ unsigned long long philox32_2(unsigned c0, unsigned c1, unsigned c2, unsigned c3,
                                                         unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const unsigned n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return ((unsigned long long)c0 << 32) | c1;
}

__device__ __forceinline__ double u01d(unsigned long long r) { return ((double)(r >> 11) + 0.5) * 0x1p-53; }
__device__ __forceinline__ float u01f(unsigned long long r) {
    return ((float)(unsigned)(r >> 41) + 0.5f) * 0x1p-23f;
}

}  // namespace dm
}  // namespace ugkwp
