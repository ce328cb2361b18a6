// Forward-mode dual numbers for the oracle's reference gradients.
//
// TEST INFRASTRUCTURE ONLY (part of the CPU oracle).  Dual<N> carries a value
// and N directional derivatives; every operation applies the chain rule
// exactly, so a function templated on its scalar type yields its derivatives
// to rounding.  The elementary functions delegate the value to the same
// routines the oracle uses for binary64 (own exp_d/log_d where the oracle uses
// them, the C library elsewhere) and differentiate analytically.
#pragma once
#include <cmath>

#include "omath.hpp"

namespace orc {

template <int N> struct Dual {
    double v = 0.0;
    double d[N] = {};
    Dual() = default;
    Dual(double x) : v(x) {}  // NOLINT: constants promote implicitly
};

template <int N> inline double value(const Dual<N>& x) { return x.v; }
inline double value(double x) { return x; }

template <int N> inline Dual<N> operator-(const Dual<N>& a) {
    Dual<N> r(-a.v);
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
}
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r(a.v + b.v);
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r(a.v - b.v);
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r(a.v * b.v);
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r(a.v / b.v);
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
    return r;
}
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) {
    Dual<N> r(a.v * b);
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b;
    return r;
}
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { return a = a + b; }
template <int N> inline Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { return a = a - b; }

template <int N> inline bool operator<(const Dual<N>& a, double b) { return a.v < b; }
template <int N> inline bool operator>(const Dual<N>& a, double b) { return a.v > b; }

// f(x) with f'(x) given: r = (f(v), f'(v) dx)
template <int N> inline Dual<N> chain(const Dual<N>& x, double f, double df) {
    Dual<N> r(f);
    for (int k = 0; k < N; ++k) r.d[k] = df * x.d[k];
    return r;
}
template <int N> inline Dual<N> sqrt(const Dual<N>& x) {
    const double s = std::sqrt(x.v);
    return chain(x, s, 0.5 / s);
}
template <int N> inline Dual<N> exp(const Dual<N>& x) {
    const double e = std::exp(x.v);
    return chain(x, e, e);
}
template <int N> inline Dual<N> expm1(const Dual<N>& x) { return chain(x, std::expm1(x.v), std::exp(x.v)); }
template <int N> inline Dual<N> erfc(const Dual<N>& x) {
    // d/dx erfc x = -2/sqrt(pi) e^{-x^2}
    return chain(x, std::erfc(x.v), -1.1283791670955126 * std::exp(-x.v * x.v));
}
template <int N> inline Dual<N> fabs(const Dual<N>& x) { return x.v < 0.0 ? -x : x; }
template <int N> inline Dual<N> pow(const Dual<N>& x, double a) {
    const double p = std::pow(x.v, a);
    return chain(x, p, a * p / x.v);
}
template <int N> inline Dual<N> exp_d(const Dual<N>& x) {
    const double e = exp_d(x.v);
    return chain(x, e, e);
}
template <int N> inline Dual<N> log_d(const Dual<N>& x) { return chain(x, log_d(x.v), 1.0 / x.v); }

}  // namespace orc
