// df64.cuh -- unevaluated sum of two floats (hi + lo, |lo| <= ulp(hi)/2),
// about 48 significant bits carried on the FP32 pipes.
//
// Error-free transformations: the sum of two floats as a float plus its
// rounding error (Knuth's TwoSum; Dekker's FastTwoSum when the first operand
// is the larger), and the product as a float plus its error from one fused
// multiply-add.  Addition follows the accurate double-word sum (two TwoSums,
// two renormalisations: relative error about 2^-46 even when the operands
// cancel), multiplication the double-word product with the cross terms added
// by FMAs (Dekker 1971; Hida, Li and Bailey 2001).  Division: one float
// quotient corrected by the df64 remainder.
//
// B300 runs FP64 at a small fraction of its FP32 rate; transforms whose
// results must hold about 1e-12 relative error run faster in df64.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace lfe {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ explicit df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit df64(int i) : df64((double)i) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ static df64 of(float f)
    {
        df64 r;
        r.hi = f;
        r.lo = 0.0f;
        return r;
    }
};

// correctly rounded float operations, never contracted into FMAs (the
// host versions serve the host-side check of these algorithms)
__host__ __device__ __forceinline__ float df_add(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    volatile float r = a + b;
    return r;
#endif
}
__host__ __device__ __forceinline__ float df_sub(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    volatile float r = a - b;
    return r;
#endif
}
__host__ __device__ __forceinline__ float df_mul(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float r = a * b;
    return r;
#endif
}
__host__ __device__ __forceinline__ float df_fma(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}
__host__ __device__ __forceinline__ float df_div(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fdiv_rn(a, b);
#else
    volatile float r = a / b;
    return r;
#endif
}

__host__ __device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e)
{
    s = df_add(a, b);
    const float bb = df_sub(s, a);
    e = df_add(df_sub(a, df_sub(s, bb)), df_sub(b, bb));
}

// |a| >= |b| (or a == 0)
__host__ __device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e)
{
    s = df_add(a, b);
    e = df_sub(b, df_sub(s, a));
}

__host__ __device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    float s1, s2, t1, t2;
    df_two_sum(a.hi, b.hi, s1, s2);
    df_two_sum(a.lo, b.lo, t1, t2);
    s2 = df_add(s2, t1);
    df_fast_two_sum(s1, s2, s1, s2);
    s2 = df_add(s2, t2);
    df64 r;
    df_fast_two_sum(s1, s2, r.hi, r.lo);
    return r;
}

__host__ __device__ __forceinline__ df64 operator-(df64 a)
{
    df64 r;
    r.hi = -a.hi;
    r.lo = -a.lo;
    return r;
}

__host__ __device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__host__ __device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = df_mul(a.hi, b.hi);
    float e = df_fma(a.hi, b.hi, -p);
    e = df_fma(a.hi, b.lo, e);
    e = df_fma(a.lo, b.hi, e);
    df64 r;
    df_fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

__host__ __device__ __forceinline__ df64 operator/(df64 a, df64 b)
{
    const float q1 = df_div(a.hi, b.hi);
    const df64 r = a - b * df64::of(q1);
    const float q2 = df_div(r.hi, b.hi);
    df64 o;
    df_fast_two_sum(q1, q2, o.hi, o.lo);
    return o;
}

__host__ __device__ __forceinline__ df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
__host__ __device__ __forceinline__ df64& operator-=(df64& a, df64 b) { a = a - b; return a; }
__host__ __device__ __forceinline__ df64& operator*=(df64& a, df64 b) { a = a * b; return a; }

}  // namespace lfe
