// Forward-mode dual numbers on the device: a value and N directional
// derivatives, each operation applying the chain rule.  The adjoint kernels
// evaluate the first-order face flux on Dual<N> to get exact local Jacobians
// (vector-Jacobian products of one face at a time).
#pragma once

namespace ugkwp {
namespace ad {

template <int N> struct Dual {
    double v;
    double d[N];
    __device__ Dual() : v(0.0) {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = 0.0;
    }
    __device__ Dual(double x) : v(x) {  // NOLINT: constants promote implicitly
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = 0.0;
    }
};

__device__ __forceinline__ double val(double x) { return x; }
template <int N> __device__ __forceinline__ double val(const Dual<N>& x) { return x.v; }

template <int N> __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
    Dual<N> r(-a.v);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r(a.v + b.v);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r(a.v - b.v);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r(a.v * b.v);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    const double ib = 1.0 / b.v;
    Dual<N> r(a.v * ib);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, double b) {
    Dual<N> r(a.v * b);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b;
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N> __device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double b) {
    Dual<N> r = a;
    r.v += b;
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator+(double a, const Dual<N>& b) { return b + a; }
template <int N> __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, double b) { return a + (-b); }
template <int N> __device__ __forceinline__ Dual<N> operator-(double a, const Dual<N>& b) { return (-b) + a; }
template <int N> __device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> __device__ __forceinline__ Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }

template <int N> __device__ __forceinline__ Dual<N> chain(const Dual<N>& x, double f, double df) {
    Dual<N> r(f);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = df * x.d[k];
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> sqrt(const Dual<N>& x) {
    const double s = ::sqrt(x.v);
    return chain(x, s, 0.5 / s);
}
template <int N> __device__ __forceinline__ Dual<N> exp(const Dual<N>& x) {
    const double e = ::exp(x.v);
    return chain(x, e, e);
}
template <int N> __device__ __forceinline__ Dual<N> log(const Dual<N>& x) { return chain(x, ::log(x.v), 1.0 / x.v); }
template <int N> __device__ __forceinline__ Dual<N> expm1(const Dual<N>& x) { return chain(x, ::expm1(x.v), ::exp(x.v)); }
template <int N> __device__ __forceinline__ Dual<N> erfc(const Dual<N>& x) {
    // d/dx erfc x = -2/sqrt(pi) e^{-x^2}
    return chain(x, ::erfc(x.v), -1.1283791670955126 * ::exp(-x.v * x.v));
}
template <int N> __device__ __forceinline__ Dual<N> fabs(const Dual<N>& x) { return x.v < 0.0 ? -x : x; }

}  // namespace ad
}  // namespace ugkwp
