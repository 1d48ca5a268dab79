// Forward-mode dual numbers in FP32: a value and K tangents.  Running the residual kernels
// on them with unit seeds in K degrees of freedom per element gives those K columns of the
// element-diagonal Jacobian block exactly (to FP32 rounding of each term), with no
// finite-difference step and no cancellation.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

// K tangent directions carried at once, so that one residual evaluation yields K columns
// of the element blocks.  K = 3 makes a 16-byte value.
template <int K>
struct __align__(16) DualN {
    float v, d[K];
    DualN() = default;
    __host__ __device__ constexpr DualN(float x) : v(x), d{} {}
    __host__ __device__ constexpr DualN(double x) : v((float)x), d{} {}
    __host__ __device__ constexpr DualN(int x) : v((float)x), d{} {}
};

#define FR_DN template <int K> __device__ __forceinline__
#define FR_EACH _Pragma("unroll") for (int t = 0; t < K; ++t)
FR_DN DualN<K> operator+(DualN<K> a, DualN<K> b) {
    DualN<K> r;
    r.v = a.v + b.v;
    FR_EACH r.d[t] = a.d[t] + b.d[t];
    return r;
}
FR_DN DualN<K> operator-(DualN<K> a, DualN<K> b) {
    DualN<K> r;
    r.v = a.v - b.v;
    FR_EACH r.d[t] = a.d[t] - b.d[t];
    return r;
}
FR_DN DualN<K> operator-(DualN<K> a) {
    DualN<K> r;
    r.v = -a.v;
    FR_EACH r.d[t] = -a.d[t];
    return r;
}
FR_DN DualN<K> operator*(DualN<K> a, DualN<K> b) {
    DualN<K> r;
    r.v = a.v * b.v;
    FR_EACH r.d[t] = fmaf(a.d[t], b.v, a.v * b.d[t]);
    return r;
}
FR_DN DualN<K> operator*(float a, DualN<K> b) {
    DualN<K> r;
    r.v = a * b.v;
    FR_EACH r.d[t] = a * b.d[t];
    return r;
}
FR_DN DualN<K> operator*(DualN<K> a, float b) { return b * a; }
FR_DN DualN<K> operator/(DualN<K> a, DualN<K> b) {
    DualN<K> r;
    float q = a.v / b.v;
    r.v = q;
    FR_EACH r.d[t] = (a.d[t] - q * b.d[t]) / b.v;
    return r;
}
FR_DN DualN<K> fma(DualN<K> a, DualN<K> b, DualN<K> c) {
    DualN<K> r;
    r.v = fmaf(a.v, b.v, c.v);
    FR_EACH r.d[t] = fmaf(a.d[t], b.v, fmaf(a.v, b.d[t], c.d[t]));
    return r;
}
FR_DN DualN<K> fma(float a, DualN<K> b, DualN<K> c) {
    DualN<K> r;
    r.v = fmaf(a, b.v, c.v);
    FR_EACH r.d[t] = fmaf(a, b.d[t], c.d[t]);
    return r;
}
FR_DN DualN<K> fma(DualN<K> a, float b, DualN<K> c) { return fma(b, a, c); }
FR_DN DualN<K> sqrt(DualN<K> a) {
    DualN<K> r;
    float s = sqrtf(a.v);
    r.v = s;
    FR_EACH r.d[t] = s > 0.f ? a.d[t] / (2.f * s) : 0.f;
    return r;
}
FR_DN DualN<K> fabs(DualN<K> a) { return a.v < 0.f ? -a : a; }
FR_DN DualN<K> fmax(DualN<K> a, DualN<K> b) { return a.v >= b.v ? a : b; }
FR_DN DualN<K> fmin(DualN<K> a, DualN<K> b) { return a.v <= b.v ? a : b; }
#undef FR_EACH
#undef FR_DN

// base type of a kernel's tables and geometric factors
template <typename T>
struct FrBase {
    typedef T type;
};
template <int K>
struct FrBase<DualN<K>> {
    typedef float type;
};
// the dual type of the FP32 element-block assembly
#define FR_AD_K 3
typedef DualN<FR_AD_K> DualT;
