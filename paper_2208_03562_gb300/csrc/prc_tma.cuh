// prc_tma.cuh -- TMA-staged persistent kernel for the interior tiles.
//
// Each CTA owns a static, strided set of W x H node tiles that lie at least two
// nodes away from every wall (no bounce-back, no ghost densities).  For each
// tile, nine tiled TMA copies (one per population plane) bring the source
// window of that plane -- the tile plus a one-node ring, shifted by -e_i --
// into shared memory, so that every pull of the tile and of the density ring
// is a shared-memory read.  Two stages: the copies of tile k+1 are in flight
// while tile k is computed.  Waits on the mbarriers are bounded; on expiry the
// CTA records LBM_ETIMEOUT in the device status, drains its own copies (again
// bounded) and returns.
#pragma once

#include <cuda.h>

#include "prc_device.cuh"
#include "prc_reduce.cuh"

namespace prc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok;
}

// Bounded wait: about two seconds of SM clock at most.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 4000000000LL) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Interior tiling: tile (tx, ty) nominally starts at (ix0 + tx W, iy0 + ty H);
// the last column / row of tiles is shifted back to start at xlast / ylast so
// that the tiles end right at the interior boundary.  Nodes of a shifted tile
// that belong to its neighbour are recomputed (identical values are stored)
// but only the owner updates the residual snapshot and the sums.
struct Interior {
    int ix0, iy0, ntx, nty;
    int xlast, ylast;
};

template <typename S, int W_, int H_>
struct TmaCfg {
    static constexpr int W = W_, H = H_;
    static constexpr int PADX = 16 / (int)sizeof(S);  // 16-byte aligned box start
    static constexpr int BW = W + 2 * PADX;           // box width (elements)
    static constexpr int BH = H + 2;                  // box height: tile + ring
    static constexpr int BOX_BYTES = BW * BH * (int)sizeof(S);
    static constexpr int PLANE_BYTES = (BOX_BYTES + 127) / 128 * 128;
    static constexpr int STAGE_BYTES = 9 * PLANE_BYTES;
    static constexpr int RW = W + 2, RH = H + 2;      // density tile with ring
    static constexpr int R_BYTES = (RW * RH * 4 + 127) / 128 * 128;
    static constexpr int SMEM = 2 * STAGE_BYTES + R_BYTES + 128 + 128;  // + barriers, + base alignment
    static constexpr int THREADS = 512;
};

template <typename S, typename T, int W, int H, bool DRHO, bool EPI>
__global__ void __launch_bounds__(512, 1)
k_step_tma(const __grid_constant__ CUtensorMap tsrc, S *__restrict__ dst, Grid gd, Coef<T> k,
           T *__restrict__ snap, double2 *__restrict__ partials, DevStatus *__restrict__ st, Interior in)
{
    using C = TmaCfg<S, W, H>;
    if (st->stop) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    S *stage0 = reinterpret_cast<S *>(smem);
    S *stage1 = reinterpret_cast<S *>(smem + C::STAGE_BYTES);
    float *R = reinterpret_cast<float *>(smem + 2 * C::STAGE_BYTES);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * C::STAGE_BYTES + C::R_BYTES);
    constexpr int PE = C::PLANE_BYTES / (int)sizeof(S);  // plane stride in elements

    const int tid = threadIdx.x;
    const int ntiles = in.ntx * in.nty;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto origin = [&](int tile, int &x0, int &y0, int &ox, int &oy) {
        ox = in.ix0 + (tile % in.ntx) * W;
        oy = in.iy0 + (tile / in.ntx) * H;
        x0 = min(ox, in.xlast);
        y0 = min(oy, in.ylast);
    };
    auto issue = [&](int tile, S *stg, uint64_t *b) {
        int x0, y0, ox, oy;
        origin(tile, x0, y0, ox, oy);
        mbar_arrive_expect_tx(b, 9u * C::BOX_BYTES);
#pragma unroll
        for (int i = 0; i < 9; i++) tma_load_3d(stg + i * PE, &tsrc, b, x0 - C::PADX, y0 - 1 - ey_of(i), i);
    };

    RedAcc<T> acc;
    int tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) issue(tile, stage0, &bar[0]);
    bool in_flight_other = false;  // (thread 0) a copy into the other stage is outstanding
    int it = 0;
    for (; tile < ntiles; it++, tile += gridDim.x) {
        const int s = it & 1;
        S *cur = s ? stage1 : stage0;
        const int next = tile + gridDim.x;
        if (tid == 0) {
            in_flight_other = next < ntiles;
            if (in_flight_other) issue(next, s ? stage0 : stage1, &bar[s ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&bar[s], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(&st->timeout, 1);
                atomicExch(&st->stop, 1);
                if (in_flight_other) mbar_wait_bounded(&bar[s ^ 1], ((it + 1) >> 1) & 1);
            }
            __syncthreads();
            return;
        }
        int x0, y0, ox, oy;
        origin(tile, x0, y0, ox, oy);

        if constexpr (DRHO) {
            // density (minus rho0) of the tile and its ring
            for (int q = tid; q < C::RW * C::RH; q += C::THREADS) {
                const int ly = q / C::RW, lx = q - ly * C::RW;  // ly, lx offset by +1
                const S *b = cur + ly * C::BW + lx - 1 + C::PADX;
                T sum = T(0);
#pragma unroll
                for (int i = 0; i < 9; i++) sum += ld_smem<S, T>(b + i * PE - ex_of(i));
                R[q] = (float)sum;
            }
            __syncthreads();
        }

        for (int q = tid; q < W * H; q += C::THREADS) {
            const int ly = q / W, lx = q - ly * W;
            const S *b = cur + (ly + 1) * C::BW + lx + C::PADX;
            T g[9];
#pragma unroll
            for (int i = 0; i < 9; i++) g[i] = ld_smem<S, T>(b + i * PE - ex_of(i));
            T dxr = T(0), dyr = T(0);
            if constexpr (DRHO) {
                const float *c = R + (ly + 1) * C::RW + (lx + 1);
                const T rE = c[1], rW = c[-1], rN = c[C::RW], rS = c[-C::RW];
                const T rNE = c[C::RW + 1], rNW = c[C::RW - 1], rSE = c[-C::RW + 1], rSW = c[-C::RW - 1];
                dxr = (T(4) * (rE - rW) + (rNE - rNW) + (rSE - rSW)) * k.inv12;
                dyr = (T(4) * (rN - rS) + (rNE - rSE) + (rNW - rSW)) * k.inv12r;
            }
            T ux, uy, drho;
            collide<T, DRHO>(k, g, dxr, dyr, ux, uy, drho);
            const long long o = (long long)(y0 + ly) * gd.pitch + (x0 + lx);
#pragma unroll
            for (int i = 0; i < 9; i++) dst[(long long)i * gd.plane + o] = to_s<S, T>(g[i]);
            if constexpr (EPI) {
                if (x0 + lx >= ox && y0 + ly >= oy) {
                    const T d = ux - snap[o];
                    snap[o] = ux;
                    acc.add(d * d, drho);
                }
            }
        }
        __syncthreads();  // stage `cur` and R are free for reuse
    }
    if constexpr (EPI) {
        __shared__ double red[2 * 16];
        double a, b;
        acc.block_total(a, b, red);
        if (tid == 0) partials[blockIdx.x] = make_double2(a, b);
    }
}

}  // namespace prc
