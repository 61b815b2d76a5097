// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits, computed on the
// FP32 pipes.  On GB300 the FP64 pipe issues about 2 FMAs per clock per SM
// against 128 FP32 FMAs, so a double-float FMA (about a dozen FP32 operations)
// is several times faster than a native double FMA, at slightly lower
// precision (relative error of each operation about 2^-44 .. 2^-48).
//
// Error-free building blocks (Knuth's TwoSum, Dekker's Fast2Sum, and the
// FMA-based exact product) follow their textbook definitions: Muller et al.,
// Handbook of Floating-Point Arithmetic, 2nd ed., Ch. 4 and Ch. 14.
#pragma once

#include <cuda_runtime.h>

namespace rbt {

struct __align__(8) df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ explicit df64(float h) : hi(h), lo(0.f) {}
    __host__ __device__ explicit df64(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
};

// s + e == a + b exactly (any magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e == a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 df_norm(float hi, float lo)
{
    df64 r;
    fast_two_sum(hi, lo, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_norm(s, e);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);   // exact error of the leading product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_norm(p, e);
}

__device__ __forceinline__ df64 operator/(df64 a, df64 b)
{
    float q1 = __fdiv_rn(a.hi, b.hi);
    df64 r = a - b * df64(q1);
    float q2 = __fdiv_rn(r.hi, b.hi);
    return df_norm(q1, q2);
}

__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator/=(df64 &a, df64 b) { return a = a / b; }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }
__device__ __forceinline__ bool isfinite(df64 a) { return ::isfinite(a.hi) && ::isfinite(a.lo); }

// Overloads for the built-in types, so that unqualified fma / isfinite in
// templated code inside namespace rbt resolve for every element type.
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fma(float a, float b, float c) { return ::fmaf(a, b, c); }
__device__ __forceinline__ bool isfinite(double a) { return ::isfinite(a); }
__device__ __forceinline__ bool isfinite(float a) { return ::isfinite(a); }

__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df64 shfl_xor(df64 v, int o)
{
    return df64(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

__device__ __forceinline__ double shfl_idx(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl_idx(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ df64 shfl_idx(df64 v, int src)
{
    return df64(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}

// loads that bypass L1 (values written by other CTAs of the same launch)
__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ df64 ld_cg(const df64 *p)
{
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return df64(v.x, v.y);
}

// conversions with double (exact split of the leading 48 bits)
__device__ __forceinline__ df64 df_from_double(double x)
{
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return df64(h, l);
}
__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

}  // namespace rbt
