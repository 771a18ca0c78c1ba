// pic_dual.cuh -- forward-mode dual numbers for the adjoint kernels.
//
// Dual<T, N> carries a value and its derivatives with respect to N seeded
// inputs.  The adjoint kernels run the forward device functions of
// pic_device.cuh (push_spin, gather_eb, deposit_esirkepov, ...) on Dual
// inputs, so every vector-Jacobian product is taken of exactly the arithmetic
// the forward step performs, branch for branch (comparisons act on values).
#pragma once
#include <cuda_runtime.h>

#include "pic_device.cuh"

template <typename T, int N>
struct Dual {
    T v;
    T d[N];
    __host__ __device__ __forceinline__ Dual() : v(T(0)) {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = T(0);
    }
    __host__ __device__ __forceinline__ Dual(T x) : v(x) {  // a constant
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = T(0);
    }
    // input number `seed` (0 <= seed < N) with value x
    __host__ __device__ __forceinline__ static Dual var(T x, int seed) {
        Dual r(x);
#pragma unroll
        for (int k = 0; k < N; ++k) r.d[k] = k == seed ? T(1) : T(0);
        return r;
    }
    __host__ __device__ __forceinline__ Dual &operator+=(const Dual &b) {
        v += b.v;
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] += b.d[k];
        return *this;
    }
    __host__ __device__ __forceinline__ Dual &operator-=(const Dual &b) {
        v -= b.v;
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] -= b.d[k];
        return *this;
    }
    __host__ __device__ __forceinline__ Dual &operator*=(const Dual &b) {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = d[k] * b.v + v * b.d[k];
        v *= b.v;
        return *this;
    }
};

template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator+(Dual<T, N> a, const Dual<T, N> &b) {
    return a += b;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator-(Dual<T, N> a, const Dual<T, N> &b) {
    return a -= b;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N> &a) {
    Dual<T, N> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator*(Dual<T, N> a, const Dual<T, N> &b) {
    return a *= b;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N> &a, const Dual<T, N> &b) {
    Dual<T, N> r;
    const T ib = T(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
// mixed with plain values
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator+(Dual<T, N> a, T b) {
    a.v += b;
    return a;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator+(T b, Dual<T, N> a) {
    a.v += b;
    return a;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator-(Dual<T, N> a, T b) {
    a.v -= b;
    return a;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator-(T b, const Dual<T, N> &a) {
    return Dual<T, N>(b) - a;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator*(Dual<T, N> a, T b) {
    a.v *= b;
#pragma unroll
    for (int k = 0; k < N; ++k) a.d[k] *= b;
    return a;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator*(T b, Dual<T, N> a) {
    return a * b;
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N> &a, T b) {
    return a * (T(1) / b);
}
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> operator/(T a, const Dual<T, N> &b) {
    return Dual<T, N>(a) / b;
}
#define PIC_DUAL_CMP(op)                                                                                  \
    template <typename T, int N>                                                                          \
    __host__ __device__ __forceinline__ bool operator op(const Dual<T, N> &a, const Dual<T, N> &b) {      \
        return a.v op b.v;                                                                                \
    }                                                                                                     \
    template <typename T, int N>                                                                          \
    __host__ __device__ __forceinline__ bool operator op(const Dual<T, N> &a, T b) {                      \
        return a.v op b;                                                                                  \
    }
PIC_DUAL_CMP(<)
PIC_DUAL_CMP(>)
PIC_DUAL_CMP(<=)
PIC_DUAL_CMP(>=)
#undef PIC_DUAL_CMP

// chain rule for a function with value f and derivative fp at a.v
template <typename T, int N>
__host__ __device__ __forceinline__ Dual<T, N> dual_apply(const Dual<T, N> &a, T f, T fp) {
    Dual<T, N> r;
    r.v = f;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = fp * a.d[k];
    return r;
}

template <typename T, int N>
struct Real<Dual<T, N>> {
    using D = Dual<T, N>;
    static __device__ __forceinline__ D rsqrt(const D &x) {
        const T r = Real<T>::rsqrt(x.v);
        return dual_apply(x, r, T(-0.5) * r * r * r);
    }
    static __device__ __forceinline__ D div(const D &a, const D &b) { return a / b; }
    static __device__ __forceinline__ D sqrt_(const D &x) {
        const T s = Real<T>::sqrt_(x.v);
        return dual_apply(x, s, T(0.5) / s);
    }
    static __device__ __forceinline__ void sincos_(const D &x, D *s, D *c) {
        T sv, cv;
        Real<T>::sincos_(x.v, &sv, &cv);
        *s = dual_apply(x, sv, cv);
        *c = dual_apply(x, cv, -sv);
    }
    static constexpr T kTaylor = Real<T>::kTaylor;
};

// value and derivatives of a Dual, as plain numbers
template <typename T, int N>
__host__ __device__ __forceinline__ T dval(const Dual<T, N> &a) {
    return a.v;
}
