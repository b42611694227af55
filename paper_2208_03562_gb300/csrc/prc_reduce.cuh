// prc_reduce.cuh -- per-CTA accumulation of the residual terms (u_x - u_x,snap)^2
// and of drho, for the FP64 residual and mass of Sec. 5.2.
//
// FP32 kernels accumulate in double-float (an FP32 sum plus an FP32 running
// error term from an exact two-sum), because FP64 arithmetic runs at a small
// fraction of the FP32 rate on this part; the per-warp totals are widened to
// FP64 and summed in a fixed order, so the result is deterministic.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace prc {

template <typename S, typename T>
__device__ __forceinline__ T ld_smem(const S *p);
template <> __device__ __forceinline__ double ld_smem<double, double>(const double *p) { return *p; }
template <> __device__ __forceinline__ float ld_smem<float, float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float ld_smem<__half, float>(const __half *p) { return __half2float(*p); }

template <typename T>
struct RedAcc;

template <>
struct RedAcc<double> {
    double a = 0.0, b = 0.0;
    __device__ __forceinline__ void add(double x, double y)
    {
        a += x;
        b += y;
    }
    // thread 0 receives the CTA totals; red holds 2 * (blockDim / 32) doubles
    __device__ __forceinline__ void block_total(double &A, double &B, double *red)
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        const int tid = threadIdx.y * blockDim.x + threadIdx.x, nw = (blockDim.x * blockDim.y) >> 5;
        if ((tid & 31) == 0) {
            red[tid >> 5] = a;
            red[nw + (tid >> 5)] = b;
        }
        __syncthreads();
        A = 0.0;
        B = 0.0;
        if (tid == 0)
            for (int w = 0; w < nw; w++) {
                A += red[w];
                B += red[nw + w];
            }
    }
};

// exact two-sum of h + v into h, error into l
__device__ __forceinline__ void df_acc(float &h, float &l, float v)
{
    const float s = h + v;
    const float bb = s - h;
    const float e = (h - (s - bb)) + (v - bb);
    h = s;
    l += e;
}

template <>
struct RedAcc<float> {
    float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
    __device__ __forceinline__ void add(float x, float y)
    {
        df_acc(ah, al, x);
        df_acc(bh, bl, y);
    }
    __device__ __forceinline__ void block_total(double &A, double &B, double *red)
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oah = __shfl_xor_sync(0xffffffffu, ah, o), oal = __shfl_xor_sync(0xffffffffu, al, o);
            const float obh = __shfl_xor_sync(0xffffffffu, bh, o), obl = __shfl_xor_sync(0xffffffffu, bl, o);
            df_acc(ah, al, oah);
            al += oal;
            df_acc(bh, bl, obh);
            bl += obl;
        }
        const int tid = threadIdx.y * blockDim.x + threadIdx.x, nw = (blockDim.x * blockDim.y) >> 5;
        if ((tid & 31) == 0) {
            red[tid >> 5] = (double)ah + (double)al;
            red[nw + (tid >> 5)] = (double)bh + (double)bl;
        }
        __syncthreads();
        A = 0.0;
        B = 0.0;
        if (tid == 0)
            for (int w = 0; w < nw; w++) {
                A += red[w];
                B += red[nw + w];
            }
    }
};

}  // namespace prc
