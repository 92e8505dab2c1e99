// lb3e_dual.cuh -- dual numbers for the tangent (forward-mode) derivative of the
// step with respect to a few model parameters.
//
// Dual<T, M> carries a value and M tangents.  Instantiating the step kernels with
// R = S = Dual<T, M> propagates d(state)/d(theta_k) exactly through every operation
// of the discrete step (chain rule per arithmetic operation), for M parameter
// directions at once; the parameters that carry tangents are injected with prm().
#pragma once

#include <cuda_runtime.h>

namespace lb3e {

template <class T, int M>
struct Dual {
    T v;
    T d[M];
    __host__ __device__ constexpr Dual() : v(0), d{} {}
    __host__ __device__ constexpr Dual(double x) : v(T(x)), d{} {}
    __host__ __device__ explicit operator double() const { return (double)v; }
};

template <class T, int M>
__host__ __device__ __forceinline__ Dual<T, M> operator+(const Dual<T, M>& a, const Dual<T, M>& b) {
    Dual<T, M> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < M; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <class T, int M>
__host__ __device__ __forceinline__ Dual<T, M> operator-(const Dual<T, M>& a, const Dual<T, M>& b) {
    Dual<T, M> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < M; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <class T, int M>
__host__ __device__ __forceinline__ Dual<T, M> operator-(const Dual<T, M>& a) {
    Dual<T, M> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < M; ++k) r.d[k] = -a.d[k];
    return r;
}
template <class T, int M>
__host__ __device__ __forceinline__ Dual<T, M> operator*(const Dual<T, M>& a, const Dual<T, M>& b) {
    Dual<T, M> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < M; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <class T, int M>
__host__ __device__ __forceinline__ Dual<T, M> operator/(const Dual<T, M>& a, const Dual<T, M>& b) {
    Dual<T, M> r;
    const T ib = T(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < M; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
template <class T, int M>
__host__ __device__ __forceinline__ Dual<T, M>& operator+=(Dual<T, M>& a, const Dual<T, M>& b) { return a = a + b; }
template <class T, int M>
__host__ __device__ __forceinline__ Dual<T, M>& operator-=(Dual<T, M>& a, const Dual<T, M>& b) { return a = a - b; }
template <class T, int M>
__host__ __device__ __forceinline__ Dual<T, M>& operator*=(Dual<T, M>& a, const Dual<T, M>& b) { return a = a * b; }

// mixed operations with plain constants (the kernels write R(c) * x; these keep
// the same meaning when a bare number meets a dual)
template <class T, int M>
__host__ __device__ __forceinline__ Dual<T, M> operator*(double a, const Dual<T, M>& b) { return Dual<T, M>(a) * b; }

template <class R> struct is_dual { static constexpr bool value = false; };
template <class T, int M> struct is_dual<Dual<T, M>> { static constexpr bool value = true; };

}  // namespace lb3e
