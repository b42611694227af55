// prc_vec.cuh -- arithmetic types of the collision: float, double, and F2, a
// pair of FP32 lanes (two neighbouring nodes) computed with the packed FP32x2
// instructions of sm_100-class GPUs (one FFMA2 / FADD2 / FMUL2 does the work of
// two scalar instructions).  The collision is written once against vadd /
// vsub / vmul / vfma / vrcp so that every type gets explicit fused
// multiply-adds.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace prc {

struct F2 {
    float2 v;
    __host__ __device__ __forceinline__ F2() {}
    __host__ __device__ __forceinline__ explicit F2(float s) : v(make_float2(s, s)) {}
    __host__ __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __host__ __device__ __forceinline__ explicit F2(float2 w) : v(w) {}
};

template <typename T> __host__ __device__ inline T from_double(double x) { return (T)x; }
template <> __host__ __device__ inline F2 from_double<F2>(double x) { return F2((float)x); }

// The helpers also compile for the host (lane-wise scalar arithmetic) so that
// the collision can be exercised off the GPU by developer tooling.
#define PRC_HD __host__ __device__ __forceinline__

// ---- scalar float.  On the device every operation is rounded on its own
// (the compiler may not fuse a product into a following sum), so that a node
// computed in a scalar lane gets bitwise what the same node gets in a packed
// FP32x2 lane, whose operations are never fused either.
PRC_HD float vadd(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
PRC_HD float vsub(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
PRC_HD float vmul(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
PRC_HD float vfma(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}
PRC_HD float vrcp(float a)
{
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
#else
    return 1.0f / a;
#endif
}

// ---- scalar double
PRC_HD double vadd(double a, double b) { return a + b; }
PRC_HD double vsub(double a, double b) { return a - b; }
PRC_HD double vmul(double a, double b) { return a * b; }
PRC_HD double vfma(double a, double b, double c)
{
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return fma(a, b, c);
#endif
}
PRC_HD double vrcp(double a) { return 1.0 / a; }

// ---- packed FP32x2
PRC_HD F2 vadd(F2 a, F2 b)
{
#ifdef __CUDA_ARCH__
    return F2(__fadd2_rn(a.v, b.v));
#else
    return F2(a.v.x + b.v.x, a.v.y + b.v.y);
#endif
}
PRC_HD F2 vmul(F2 a, F2 b)
{
#ifdef __CUDA_ARCH__
    return F2(__fmul2_rn(a.v, b.v));
#else
    return F2(a.v.x * b.v.x, a.v.y * b.v.y);
#endif
}
PRC_HD F2 vfma(F2 a, F2 b, F2 c)
{
#ifdef __CUDA_ARCH__
    return F2(__ffma2_rn(a.v, b.v, c.v));
#else
    return F2(fmaf(a.v.x, b.v.x, c.v.x), fmaf(a.v.y, b.v.y, c.v.y));
#endif
}
// a - b = b * (-1) + a, exact like a scalar subtraction
PRC_HD F2 vsub(F2 a, F2 b) { return vfma(b, F2(-1.f), a); }
PRC_HD F2 vrcp(F2 a) { return F2(vrcp(a.v.x), vrcp(a.v.y)); }

template <typename T> struct Lane { using type = T; };
template <> struct Lane<F2> { using type = float; };

template <typename T>
PRC_HD T splat(double s) { return T(s); }
template <>
PRC_HD F2 splat<F2>(double s) { return F2((float)s); }

}  // namespace prc
