// Oracle-side elementary functions and counter-based random numbers.
//
// TEST INFRASTRUCTURE ONLY: part of the plain CPU oracle of the UGKWP step.
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
// load it; the product path never does.
//
// The particle path of the method must be reproducible bit for bit on any
// IEEE-754 machine, so the transcendental functions it needs are written
// here from textbook methods using only +, -, *, / and sqrt (all correctly
// rounded) with floating-point contraction disabled (-ffp-contract=off):
//
//   exp_d     Cody-Waite reduction x = k ln2 + r with a two-part ln2, then the
//             degree-13 Taylor polynomial of e^r (|r| <= ln2/2) and a power-of-
//             two scaling.  Truncation error r^14/14! < 4e-18.
//   log_d     x = 2^e m with m in (sqrt(1/2), sqrt(2)], f = (m-1)/(m+1),
//             log m = 2 atanh f = 2 (f + f^3/3 + ... + f^23/23), |f| < 0.172.
//   log_f     the same identity in binary32 (series up to f^11/11).
//   sincos2pi sin/cos of 2*pi*u: exact reduction by quarter turns (4u - j),
//             then Taylor series of sin and cos on [-pi/4, pi/4]; sincos2pi_f
//             the same in binary32 (sin to th^11/11!, cos to th^12/12!).
//   philox    Philox4x64-10 and Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
//             "Parallel random numbers: as easy as 1, 2, 3", SC'11): 10 rounds of
//             two multiplies (64x64->128, resp. 32x32->64) with the published
//             multipliers and Weyl key bumps.
//
// Constants are hexadecimal literals of the exact rationals they stand for
// (1/k!, 1/(2k+1), ln2 split into a 32-bit head and a tail, pi/2).
#pragma once
#include <cstdint>
#include <cstring>
#include <cmath>

namespace orc {

inline double bits_to_double(uint64_t b) { double d; std::memcpy(&d, &b, 8); return d; }
inline uint64_t double_to_bits(double d) { uint64_t b; std::memcpy(&b, &d, 8); return b; }
inline float bits_to_float(uint32_t b) { float f; std::memcpy(&f, &b, 4); return f; }
inline uint32_t float_to_bits(float f) { uint32_t b; std::memcpy(&b, &f, 4); return b; }

// 2^k as a double for -1022 <= k <= 1023 (exact).
inline double pow2i(int k) { return bits_to_double((uint64_t)(k + 1023) << 52); }

// ---------------------------------------------------------------- exp(x)
inline double exp_d(double x) {
    if (x != x) return x;
    if (x > 709.782712893384) return HUGE_VAL;
    if (x < -745.2) return 0.0;
    const double INV_LN2 = 0x1.71547652b82fep+0;
    const double LN2_HI = 0x1.62e42fee00000p-1;   // ln2 truncated to 32 bits
    const double LN2_LO = 0x1.a39ef35793c76p-33;  // ln2 - LN2_HI
    double k = std::floor(x * INV_LN2 + 0.5);
    double r = (x - k * LN2_HI) - k * LN2_LO;
    // Horner evaluation of sum_{j=0}^{13} r^j / j!
    double p = 0x1.6124613a86d09p-33;             // 1/13!
    p = p * r + 0x1.1eed8eff8d898p-29;            // 1/12!
    p = p * r + 0x1.ae64567f544e4p-26;            // 1/11!
    p = p * r + 0x1.27e4fb7789f5cp-22;            // 1/10!
    p = p * r + 0x1.71de3a556c734p-19;            // 1/9!
    p = p * r + 0x1.a01a01a01a01ap-16;            // 1/8!
    p = p * r + 0x1.a01a01a01a01ap-13;            // 1/7!
    p = p * r + 0x1.6c16c16c16c17p-10;            // 1/6!
    p = p * r + 0x1.1111111111111p-7;             // 1/5!
    p = p * r + 0x1.5555555555555p-5;             // 1/4!
    p = p * r + 0x1.5555555555555p-3;             // 1/3!
    p = p * r + 0x1.0000000000000p-1;             // 1/2!
    p = p * r + 1.0;
    p = p * r + 1.0;
    int ki = (int)k;
    if (ki > 1023) return (p * pow2i(ki - 1)) * 2.0;
    if (ki >= -1022) return p * pow2i(ki);
    return (p * pow2i(ki + 60)) * pow2i(-60);     // gradual underflow: one rounding
}

// ---------------------------------------------------------------- log(x)
inline double log_d(double x) {
    if (x != x || x < 0.0) return NAN;
    if (x == 0.0) return -HUGE_VAL;
    if (std::isinf(x)) return x;
    int e_adj = 0;
    if (x < 0x1p-1022) { x = x * 0x1p54; e_adj = -54; }   // subnormal input
    uint64_t b = double_to_bits(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = bits_to_double((b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL);  // [1,2)
    if (m > 0x1.6a09e667f3bcdp+0) { m = m * 0.5; e += 1; }   // m in (sqrt(1/2), sqrt(2)]
    e += e_adj;
    double f = (m - 1.0) / (m + 1.0);
    double s = f * f;
    // sum_{j=0}^{11} s^j / (2j+1)
    double q = 0x1.642c8590b2164p-5;              // 1/23
    q = q * s + 0x1.8618618618618p-5;             // 1/21
    q = q * s + 0x1.af286bca1af28p-5;             // 1/19
    q = q * s + 0x1.e1e1e1e1e1e1ep-5;             // 1/17
    q = q * s + 0x1.1111111111111p-4;             // 1/15
    q = q * s + 0x1.3b13b13b13b14p-4;             // 1/13
    q = q * s + 0x1.745d1745d1746p-4;             // 1/11
    q = q * s + 0x1.c71c71c71c71cp-4;             // 1/9
    q = q * s + 0x1.2492492492492p-3;             // 1/7
    q = q * s + 0x1.999999999999ap-3;             // 1/5
    q = q * s + 0x1.5555555555555p-2;             // 1/3
    double f2 = f + f;
    double logm = f2 + (f2 * s) * q;
    const double LN2_HI = 0x1.62e42fee00000p-1;
    const double LN2_LO = 0x1.a39ef35793c76p-33;
    double de = (double)e;
    return de * LN2_HI + (de * LN2_LO + logm);
}

// ---------------------------------------------------------------- logf(x)
inline float log_f(float x) {
    if (x != x || x < 0.0f) return NAN;
    if (x == 0.0f) return -HUGE_VALF;
    if (std::isinf(x)) return x;
    int e_adj = 0;
    if (x < 0x1p-126f) { x = x * 0x1p24f; e_adj = -24; }
    uint32_t b = float_to_bits(x);
    int e = (int)((b >> 23) & 0xff) - 127;
    float m = bits_to_float((b & 0x007fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) { m = m * 0.5f; e += 1; }
    e += e_adj;
    float f = (m - 1.0f) / (m + 1.0f);
    float s = f * f;
    float q = 0x1.745d18p-4f;                     // 1/11
    q = q * s + 0x1.c71c72p-4f;                   // 1/9
    q = q * s + 0x1.24924ap-3f;                   // 1/7
    q = q * s + 0x1.99999ap-3f;                   // 1/5
    q = q * s + 0x1.555556p-2f;                   // 1/3
    float f2 = f + f;
    float logm = f2 + (f2 * s) * q;
    const float LN2_HI = 0x1.62e4p-1f;            // ln2 truncated to 16 bits
    const float LN2_LO = 0x1.7f7d1cp-20f;         // ln2 - LN2_HI
    float de = (float)e;
    return de * LN2_HI + (de * LN2_LO + logm);
}

// ------------------------------------------------- sin(2 pi u), cos(2 pi u)
inline void sincos2pi_d(double u, double* s_out, double* c_out) {
    double q = 4.0 * u;                            // quarter turns (exact)
    double j = std::floor(q + 0.5);
    double r = q - j;                              // exact, |r| <= 1/2
    double th = r * 0x1.921fb54442d18p+0;          // r * pi/2, |th| <= pi/4
    double t2 = th * th;
    // sin th = th * sum_{k=0}^{9} (-1)^k th^{2k} / (2k+1)!
    double ps = -0x1.2f49b46814157p-57;            // -1/19!
    ps = ps * t2 + 0x1.952c77030ad4ap-49;          // +1/17!
    ps = ps * t2 - 0x1.ae7f3e733b81fp-41;          // -1/15!
    ps = ps * t2 + 0x1.6124613a86d09p-33;          // +1/13!
    ps = ps * t2 - 0x1.ae64567f544e4p-26;          // -1/11!
    ps = ps * t2 + 0x1.71de3a556c734p-19;          // +1/9!
    ps = ps * t2 - 0x1.a01a01a01a01ap-13;          // -1/7!
    ps = ps * t2 + 0x1.1111111111111p-7;           // +1/5!
    ps = ps * t2 - 0x1.5555555555555p-3;           // -1/3!
    double sn = th + (th * t2) * ps;
    // cos th = sum_{k=0}^{10} (-1)^k th^{2k} / (2k)!
    double pc = 0x1.e542ba4020225p-62;             // +1/20!
    pc = pc * t2 - 0x1.6827863b97d97p-53;          // -1/18!
    pc = pc * t2 + 0x1.ae7f3e733b81fp-45;          // +1/16!
    pc = pc * t2 - 0x1.93974a8c07c9dp-37;          // -1/14!
    pc = pc * t2 + 0x1.1eed8eff8d898p-29;          // +1/12!
    pc = pc * t2 - 0x1.27e4fb7789f5cp-22;          // -1/10!
    pc = pc * t2 + 0x1.a01a01a01a01ap-16;          // +1/8!
    pc = pc * t2 - 0x1.6c16c16c16c17p-10;          // -1/6!
    pc = pc * t2 + 0x1.5555555555555p-5;           // +1/4!
    pc = pc * t2 - 0x1.0000000000000p-1;           // -1/2!
    double cs = 1.0 + t2 * pc;
    int quadrant = ((int)j) & 3;
    switch (quadrant) {
        case 0: *s_out = sn;  *c_out = cs;  break;
        case 1: *s_out = cs;  *c_out = -sn; break;
        case 2: *s_out = -sn; *c_out = -cs; break;
        default: *s_out = -cs; *c_out = sn; break;
    }
}

// Binary32 variant for particles of the mixed-precision mode.  4u and q - j
// are exact for u on the 2^-24 grid of u01_f; |th| <= pi/4 in binary32 with
// truncation errors th^13/13! and th^14/14! below 1e-11.
inline void sincos2pi_f(float u, float* s_out, float* c_out) {
    float q = 4.0f * u;
    float j = std::floor(q + 0.5f);
    float th = (q - j) * 0x1.921fb6p+0f;           // pi/2 in binary32
    float t2 = th * th;
    float ps = -0x1.ae6456p-26f;                   // -1/11!
    ps = ps * t2 + 0x1.71de3ap-19f;                // +1/9!
    ps = ps * t2 - 0x1.a01a02p-13f;                // -1/7!
    ps = ps * t2 + 0x1.111112p-7f;                 // +1/5!
    ps = ps * t2 - 0x1.555556p-3f;                 // -1/3!
    float sn = th + (th * t2) * ps;
    float pc = 0x1.1eed8ep-29f;                    // +1/12!
    pc = pc * t2 - 0x1.27e4fcp-22f;                // -1/10!
    pc = pc * t2 + 0x1.a01a02p-16f;                // +1/8!
    pc = pc * t2 - 0x1.6c16c2p-10f;                // -1/6!
    pc = pc * t2 + 0x1.555556p-5f;                 // +1/4!
    pc = pc * t2 - 0x1p-1f;                        // -1/2!
    float cs = 1.0f + t2 * pc;
    int quadrant = ((int)j) & 3;
    switch (quadrant) {
        case 0: *s_out = sn;  *c_out = cs;  break;
        case 1: *s_out = cs;  *c_out = -sn; break;
        case 2: *s_out = -sn; *c_out = -cs; break;
        default: *s_out = -cs; *c_out = sn; break;
    }
}

// ------------------------------------------------------------ Philox4x64-10
struct Ctr4 { uint64_t v[4]; };

inline Ctr4 philox4x64_10(Ctr4 c, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)M0 * c.v[0];
        unsigned __int128 p1 = (unsigned __int128)M1 * c.v[2];
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        Ctr4 n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
        k0 += W0; k1 += W1;
    }
    return c;
}

// Philox4x32-10 (same paper): 10 rounds of two 32x32->64 multiplies with the
// published multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key bumps 0x9E3779B9,
// 0xBB67AE85.  Used for the free-transport-time draw, the one draw per particle
// and step on the tracking path.
struct Ctr4x32 { uint32_t v[4]; };

inline Ctr4x32 philox4x32_10(Ctr4x32 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * c.v[0];
        uint64_t p1 = (uint64_t)M1 * c.v[2];
        Ctr4x32 n;
        n.v[0] = (uint32_t)(p1 >> 32) ^ c.v[1] ^ k0;
        n.v[1] = (uint32_t)p1;
        n.v[2] = (uint32_t)(p0 >> 32) ^ c.v[3] ^ k1;
        n.v[3] = (uint32_t)p0;
        c = n;
        k0 += W0; k1 += W1;
    }
    return c;
}

// Uniform on the open interval (0,1) from 64 random bits: 53-bit grid, midpoint.
inline double u01_d(uint64_t r) { return ((double)(r >> 11) + 0.5) * 0x1p-53; }
// Binary32 variant: 23-bit grid, midpoint (exactly representable).
inline float u01_f(uint64_t r) { return ((float)(uint32_t)(r >> 41) + 0.5f) * 0x1p-23f; }

}  // namespace orc
