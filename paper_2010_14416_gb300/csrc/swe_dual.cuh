// swe_dual.cuh -- forward-mode dual numbers for the discrete adjoint.
//
// Dual<N> carries a value and N directional derivatives.  Comparisons look
// at the value only, so a templated kernel function run on duals takes the
// same branches as on plain doubles and yields the derivative of the branch
// taken (for max(a, b) with a tie, the branch the code selects).
#pragma once

#include <cuda_runtime.h>

#include "swe_kernels.cuh"

namespace swe {

template <int N>
struct Dual {
    double v;
    double d[N];
    __device__ __forceinline__ Dual() : v(0.0) {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = 0.0;
    }
    __device__ __forceinline__ Dual(double x) : v(x) {  // NOLINT: implicit from constants
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = 0.0;
    }
    static __device__ __forceinline__ Dual seed(double x, int k) {
        Dual r(x);
        r.d[k] = 1.0;
        return r;
    }
};

template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
    Dual<N> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
// a / b: one division (1/b, which the derivative needs anyway) and a
// multiplication for the value; the value may differ from the quotient
// rounded once by an ulp, which the derivative does not notice.
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    const double rb = 1.0 / b.v;
    const double q = a.v * rb;
    r.v = q;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - q * b.d[k]) * rb;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { return a = a + b; }

template <int N> __device__ __forceinline__ bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N> __device__ __forceinline__ bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }
template <int N> __device__ __forceinline__ bool operator<=(const Dual<N>& a, const Dual<N>& b) { return a.v <= b.v; }
template <int N> __device__ __forceinline__ bool operator>=(const Dual<N>& a, const Dual<N>& b) { return a.v >= b.v; }

template <int N>
struct Ar<Dual<N>> {
    using D = Dual<N>;
    static __device__ __forceinline__ D sqrt_(const D& x) {
        D r;
        r.v = sqrt(x.v);
        const double k = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) r.d[j] = k * x.d[j];
        return r;
    }
    static __device__ __forceinline__ D rsqrt_(const D& x) {
        D r;
        r.v = 1.0 / sqrt(x.v);
        const double k = -0.5 * r.v / x.v;
#pragma unroll
        for (int j = 0; j < N; ++j) r.d[j] = k * x.d[j];
        return r;
    }
    static __device__ __forceinline__ D div_(const D& a, const D& b) { return a / b; }
    static __device__ __forceinline__ D rcp_(const D& x) { return D(1.0) / x; }
    static __device__ __forceinline__ D pow_m73(const D& h) {
        D r;
        r.v = 1.0 / (h.v * h.v * cbrt(h.v));
        const double k = -(7.0 / 3.0) * r.v / h.v;
#pragma unroll
        for (int j = 0; j < N; ++j) r.d[j] = k * h.d[j];
        return r;
    }
};

}  // namespace swe
