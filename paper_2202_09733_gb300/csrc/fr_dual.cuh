// Forward-mode dual number {value, derivative} in FP32.  Running the residual kernels on
// DualF with a unit seed in one degree of freedom per element gives that column of the
// element-diagonal Jacobian block exactly (to FP32 rounding of each term), with no
// finite-difference step and no cancellation.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

struct DualF {
    float v, d;
    DualF() = default;
    __host__ __device__ constexpr DualF(float x) : v(x), d(0.f) {}
    __host__ __device__ constexpr DualF(double x) : v((float)x), d(0.f) {}
    __host__ __device__ constexpr DualF(int x) : v((float)x), d(0.f) {}
    __host__ __device__ constexpr DualF(float x, float dx) : v(x), d(dx) {}
};

__device__ __forceinline__ DualF operator+(DualF a, DualF b) { return DualF(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ DualF operator-(DualF a, DualF b) { return DualF(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ DualF operator-(DualF a) { return DualF(-a.v, -a.d); }
__device__ __forceinline__ DualF operator*(DualF a, DualF b) { return DualF(a.v * b.v, fmaf(a.d, b.v, a.v * b.d)); }
__device__ __forceinline__ DualF operator*(float a, DualF b) { return DualF(a * b.v, a * b.d); }
__device__ __forceinline__ DualF operator*(DualF a, float b) { return DualF(a.v * b, a.d * b); }
__device__ __forceinline__ DualF operator/(DualF a, DualF b) {
    float q = a.v / b.v;
    return DualF(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ DualF fma(DualF a, DualF b, DualF c) {
    return DualF(fmaf(a.v, b.v, c.v), fmaf(a.d, b.v, fmaf(a.v, b.d, c.d)));
}
__device__ __forceinline__ DualF fma(float a, DualF b, DualF c) { return DualF(fmaf(a, b.v, c.v), fmaf(a, b.d, c.d)); }
__device__ __forceinline__ DualF fma(DualF a, float b, DualF c) { return DualF(fmaf(a.v, b, c.v), fmaf(a.d, b, c.d)); }
__device__ __forceinline__ DualF sqrt(DualF a) {
    float s = sqrtf(a.v);
    return DualF(s, s > 0.f ? a.d / (2.f * s) : 0.f);
}
__device__ __forceinline__ DualF fabs(DualF a) { return a.v < 0.f ? -a : a; }
__device__ __forceinline__ DualF fmax(DualF a, DualF b) { return a.v >= b.v ? a : b; }

// base type of a kernel's tables and geometric factors
template <typename T>
struct FrBase {
    typedef T type;
};
template <>
struct FrBase<DualF> {
    typedef float type;
};
