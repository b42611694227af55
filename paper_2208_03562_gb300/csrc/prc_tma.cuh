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
#include "prc_kernels.cuh"
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

// Tiled TMA store of a box from shared memory (bulk-group completion), and
// the bulk-group bookkeeping around it.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int c0, int c1, int c2)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// every committed store has finished reading its shared-memory source
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store is complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// make this thread's shared-memory writes visible to the async (TMA) proxy
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Interior tiling: tile (tx, ty) nominally starts at (ix0 + tx W, iy0 + ty H);
// the last column / row of tiles is shifted back to start at xlast / ylast so
// that the tiles end right at the interior boundary.  Nodes of a shifted tile
// that belong to its neighbour are recomputed (identical values are stored)
// but only the owner updates the residual snapshot and the sums.
struct Interior {
    int ix0, iy0, ntx, nty;
    int xlast, ylast;
    int rev;  // take the tiles in reverse order (alternate steps, see k_step_tma)
};

template <typename S, int W_, int H_, int THREADS_ = 512>
struct TmaCfg {
    static constexpr int W = W_, H = H_;
    static constexpr int PADX = 16 / (int)sizeof(S);  // 16-byte aligned box start
    static constexpr int BW = W + 2 * PADX;           // box width (elements)
    static constexpr int BH = H + 2;                  // box height: tile + ring
    static constexpr int BOX_BYTES = BW * BH * (int)sizeof(S);
    static constexpr int PLANE_BYTES = (BOX_BYTES + 127) / 128 * 128;
    static constexpr int STAGE_BYTES = 9 * PLANE_BYTES;
    static constexpr int RW = W + 4, RH = H + 2;      // density tile: node lx at column lx + 2
    static constexpr int R_BYTES = (RW * RH * 4 + 127) / 128 * 128;
    // FP16 storage writes each tile through a shared output tile and TMA
    // stores (two buffers); FP32 stores straight from registers
    static constexpr bool TSTORE = sizeof(S) == 2;
    static constexpr int OUT_PLANE = W * H * (int)sizeof(S);  // bytes of one plane of the output tile
    static constexpr int OUT_BYTES = TSTORE ? 9 * OUT_PLANE : 0;
    static constexpr int SMEM = 2 * STAGE_BYTES + 2 * R_BYTES + 2 * OUT_BYTES + 128 + 128;  // + barriers, + base alignment
    static constexpr int THREADS = THREADS_;
    static constexpr int PAIRS = W / 2;               // node pairs per tile row
    static constexpr int NQ = H * PAIRS / THREADS;    // node pairs per thread per tile
};

// Shared-memory access to a pair of neighbouring nodes (x, x+1) of one plane.
template <typename S>
struct Pair;
template <>
struct Pair<float> {
    static __device__ __forceinline__ F2 aligned(const float *p) { return F2(*reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ F2 any(const float *p) { return F2(p[0], p[1]); }
    static __device__ __forceinline__ float one(const float *p) { return *p; }
    static __device__ __forceinline__ void store(float *p, F2 v) { *reinterpret_cast<float2 *>(p) = v.v; }
};
template <>
struct Pair<__half> {
    static __device__ __forceinline__ F2 aligned(const __half *p)
    {
        return F2(__half22float2(*reinterpret_cast<const __half2 *>(p)));
    }
    static __device__ __forceinline__ F2 any(const __half *p) { return F2(__half2float(p[0]), __half2float(p[1])); }
    static __device__ __forceinline__ float one(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void store(__half *p, F2 v)
    {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.v.x, v.v.y);
    }
};

// The nine pulled values of the node pair whose first node sits at element
// `b` of plane 0 (ring-relative addressing: pull from plane i at b + i PE - e_ix).
template <typename S, int PE>
__device__ __forceinline__ void pull_pair(const S *b, F2 g[9])
{
#pragma unroll
    for (int i = 0; i < 9; i++) {
        if (ex_of(i) == 0) g[i] = Pair<S>::aligned(b + i * PE);
        else g[i] = Pair<S>::any(b + i * PE - ex_of(i));
    }
}

// Density (minus rho0) of one ring unit of a staged W x H tile, for the
// first 2 (W/2) + 2 (H + 2) threads: a pair of the row below or above the
// tile, or one node of the column left or right of it, into the density tile
// Rs (node lx of tile row ly at Rs[(ly + 1) RW + lx + 2]).  The same
// summation order as every other density, so a node's density does not
// depend on which tile formed it.
template <typename S, int W, int H, int PE, int BW, int RW, int PADX>
__device__ __forceinline__ void ring_density(int tid, const S *cur, float *Rs)
{
    constexpr int PAIRS = W / 2;
    if (tid < 2 * PAIRS) {
        const int ry = tid < PAIRS ? 0 : H + 1;
        const int rx = 2 * (tid < PAIRS ? tid : tid - PAIRS);
        F2 gr[9];
        pull_pair<S, PE>(cur + ry * BW + rx + PADX, gr);
        *reinterpret_cast<float2 *>(Rs + ry * RW + rx + 2) = sum9(gr).v;
    } else {
        const int c = tid - 2 * PAIRS;
        const int ry = c >> 1, lx = (c & 1) ? W : -1;
        const S *b = cur + ry * BW + lx + PADX;
        float gr[9];
#pragma unroll
        for (int i = 0; i < 9; i++) gr[i] = Pair<S>::one(b + i * PE - ex_of(i));
        Rs[ry * RW + lx + 2] = sum9(gr);
    }
}

// Density gradients (reading A1) of the node pair whose first node's density
// sits at c = Rs + (ly + 1) RW + x + 2 of a density tile with rows of RW.
template <int RW>
__device__ __forceinline__ void pair_gradients(const float *c, float i12, float i12r, F2 &dxr, F2 &dyr)
{
    const float2 L = *reinterpret_cast<const float2 *>(c - 2), M = *reinterpret_cast<const float2 *>(c),
                 Rr = *reinterpret_cast<const float2 *>(c + 2);
    const float2 NL = *reinterpret_cast<const float2 *>(c + RW - 2),
                 NM = *reinterpret_cast<const float2 *>(c + RW),
                 NR = *reinterpret_cast<const float2 *>(c + RW + 2);
    const float2 SL = *reinterpret_cast<const float2 *>(c - RW - 2),
                 SM = *reinterpret_cast<const float2 *>(c - RW),
                 SR = *reinterpret_cast<const float2 *>(c - RW + 2);
    // node x: E = M.y, W = L.y, N = NM.x, S = SM.x, NE = NM.y, NW = NL.y, SE = SM.y, SW = SL.y
    // node x+1: E = Rr.x, W = M.x, N = NM.y, S = SM.y, NE = NR.x, NW = NM.x, SE = SR.x, SW = SM.x
    drho_stencil<F2>(F2(M.y, Rr.x), F2(L.y, M.x), F2(NM.x, NM.y), F2(SM.x, SM.y), F2(NM.y, NR.x), F2(NL.y, NM.x),
                     F2(SM.y, SR.x), F2(SL.y, SM.x), F2(i12), F2(i12r), dxr, dyr);
}

// Persistent step kernel: the interior tiles, NQ pairs of neighbouring nodes
// per thread (rows ly, ly + H/NQ, ...; H W / 2 = NQ THREADS) with the
// collision in packed FP32x2 arithmetic, then the edge strips (`edge`,
// general tile body with bounce-back and the lid, plain loads), so that one
// launch is one time step.
//
// FP16 storage: the collided pairs go to a shared output tile (two buffers,
// alternating by tile), and the producer writes a tile with nine tiled TMA stores
// right after the next tile's barrier (every thread has written and fenced
// its part by then); before a buffer is refilled, the producer waits until the
// stores issued from it have read it.  This replaces nine global stores and
// their 64-bit address arithmetic per pair with shared-memory stores at fixed
// offsets.  FP32 storage stores from registers (its shared memory is taken by
// the wider staging windows).
//
// Per tile: every thread pulls its pairs from the staged planes once and
// keeps the nine values of each in registers; the density of the pairs (and
// of one ring unit for the first 2 W/2 + 2 (H + 2) threads) goes to the
// density tile R[it & 1]; after one barrier the thread forms the density
// gradients from R[it & 1] and collides its pairs.  That barrier is the only
// one per tile: after it the stage just read is free, so the producer refills it
// with the copies of the tile after next (two tiles in flight during the
// collision), and the density tile alternates between two buffers, so a
// thread may start the next tile while others still read this tile's
// densities (the next write of R[it & 1] comes after the next barrier, which
// every thread reaches only once its collision of this tile is done).  The
// producer is lane 0 of the last warp, which forms no ring densities, so that
// its copies and stores do not add to the ring warps' share of a tile.
template <typename S, int W, int H, int THREADS, int MINB, bool DRHO, bool EPI, bool FORCE>
__global__ void __launch_bounds__(THREADS, MINB)
k_step_tma(const __grid_constant__ CUtensorMap tsrc, const __grid_constant__ CUtensorMap tdst,
           const S *__restrict__ src, S *__restrict__ dst, Grid gd,
           Coef<F2> k, Coef<float> kf, float *__restrict__ snap, double2 *__restrict__ partials,
           DevStatus *__restrict__ st, Interior in, const __grid_constant__ Rects edge)
{
    using C = TmaCfg<S, W, H, THREADS>;
    static_assert(C::NQ >= 1 && C::NQ * THREADS == H * C::PAIRS, "whole node pairs per thread");
    static_assert(2 * C::PAIRS + 2 * C::RH <= THREADS - 32, "one ring unit per thread at most, none in the producer's warp");
    static_assert(C::R_BYTES >= srho_floats(THREADS) * (int)sizeof(float), "density tile too small for the strips");
    static_assert(C::OUT_PLANE % 128 == 0, "TMA store sources start on 128-byte boundaries");
    if (st->stop) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned base; offsetting the shared array (rather than casting
    // through an integer) keeps the accesses in the shared address space
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    S *stage0 = reinterpret_cast<S *>(smem);
    S *stage1 = reinterpret_cast<S *>(smem + C::STAGE_BYTES);
    float *R = reinterpret_cast<float *>(smem + 2 * C::STAGE_BYTES);
    S *out0 = reinterpret_cast<S *>(smem + 2 * C::STAGE_BYTES + 2 * C::R_BYTES);
    S *out1 = reinterpret_cast<S *>(smem + 2 * C::STAGE_BYTES + 2 * C::R_BYTES + C::OUT_BYTES);
    constexpr int OPE = C::OUT_PLANE / (int)sizeof(S);  // elements per output-tile plane
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * C::STAGE_BYTES + 2 * C::R_BYTES + 2 * C::OUT_BYTES);
    constexpr int RF = C::R_BYTES / (int)sizeof(float);  // floats per density tile
    constexpr int PE = C::PLANE_BYTES / (int)sizeof(S);  // plane stride in elements
    constexpr int RING = 2 * C::PAIRS + 2 * C::RH;        // ring units: 2 rows of pairs, 2 columns

    const int tid = threadIdx.x;
    constexpr int PROD = THREADS - 32;
    // this thread's pairs in the tile: column x, rows ly0 + j H / NQ
    const int ly0 = tid / C::PAIRS, x = 2 * (tid - ly0 * C::PAIRS);
    constexpr int DY = H / C::NQ;
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

    // Alternate steps take the tiles in opposite orders, so that a step first
    // reads what the previous one wrote last, while it is still in L2.  `tile`
    // runs over positions in the order; order(q) is the tile at position q.
    auto order = [&](int q) { return in.rev ? ntiles - 1 - q : q; };
    RedAcc<float> acc;
    int tile = blockIdx.x;
    if (tid == PROD) {
        if (tile < ntiles) issue(order(tile), stage0, &bar[0]);
        if (tile + (int)gridDim.x < ntiles) issue(order(tile + gridDim.x), stage1, &bar[1]);
    }
    // tile coordinates of this CTA's current tile, advanced by gridDim.x
    // tiles per iteration without a division
    const int first = order(blockIdx.x);
    int tcx = first % in.ntx, tcy = first / in.ntx;
    const int sdx = gridDim.x % in.ntx, sdy = gridDim.x / in.ntx;
    int px0 = 0, py0 = 0;  // origin of the previous tile (its TMA store is issued one tile later)
    int it = 0;
    for (; tile < ntiles; it++, tile += gridDim.x) {
        const int s = it & 1;
        S *cur = s ? stage1 : stage0;
        float *Rs = R + s * RF;
        const int ox = in.ix0 + tcx * W, oy = in.iy0 + tcy * H;
        const int x0 = min(ox, in.xlast), y0 = min(oy, in.ylast);
        if (!in.rev) {
            tcx += sdx;
            tcy += sdy;
            if (tcx >= in.ntx) {
                tcx -= in.ntx;
                tcy++;
            }
        } else {
            tcx -= sdx;
            tcy -= sdy;
            if (tcx < 0) {
                tcx += in.ntx;
                tcy--;
            }
        }
        const bool own_x = x0 + x >= ox;  // the pair's column is owned by this tile
        float2 snv[C::NQ];
        if constexpr (EPI) {
            // the snapshot is touched once per residual step: stream it, and
            // issue the loads now so that they overlap the copies
#pragma unroll
            for (int j = 0; j < C::NQ; j++) {
                const int ly = ly0 + j * DY;
                snv[j] = make_float2(0.f, 0.f);
                if (own_x & (y0 + ly >= oy))
                    snv[j] = __ldcs(reinterpret_cast<const float2 *>(snap + (long long)(y0 + ly) * gd.pitch + x0 + x));
            }
        }
        // A thread whose wait runs out still pulls (stale shared memory, no
        // harm) so that every thread reaches the one barrier of the tile,
        // which also takes the vote: on a timeout anywhere the CTA leaves
        // there, before any store of this tile.
        const bool ok = mbar_wait_bounded(&bar[s], (it >> 1) & 1);

        F2 g[C::NQ][9];
#pragma unroll
        for (int j = 0; j < C::NQ; j++) pull_pair<S, PE>(cur + (ly0 + j * DY + 1) * C::BW + x + C::PADX, g[j]);
        if constexpr (DRHO) {
            // density (minus rho0) of the pairs, and of one ring unit
#pragma unroll
            for (int j = 0; j < C::NQ; j++)
                *reinterpret_cast<float2 *>(Rs + (ly0 + j * DY + 1) * C::RW + x + 2) = sum9(g[j]).v;
            if (tid < RING) ring_density<S, W, H, PE, C::BW, C::RW, C::PADX>(tid, cur, Rs);
        }
        if constexpr (C::TSTORE) {
            // the store of tile it - 2 (issued one tile ago) has read its
            // output buffer, which this tile's collision refills
            if (tid == PROD) bulk_wait_read_all();
        }
        // FP16 storage: the half of the collision that needs no density
        // gradient runs before the barrier, while the warps with ring
        // densities to form are still at it
        Moments<F2> mom[C::NQ];
        if constexpr (C::TSTORE) {
#pragma unroll
            for (int j = 0; j < C::NQ; j++) collide_moments<F2, FORCE>(k, g[j], mom[j]);
        }
        // every pull from `cur` is done and R[s] is complete
        if (__syncthreads_or(!ok)) {
            if (tid == PROD) {
                atomicExch(&st->timeout, 1);
                atomicExch(&st->stop, 1);
                // the copies of the next tile into the other stage may be outstanding
                if (tile + (int)gridDim.x < ntiles) mbar_wait_bounded(&bar[s ^ 1], ((it + 1) >> 1) & 1);
                if constexpr (C::TSTORE) bulk_wait_all();
            }
            return;
        }
        if (tid == PROD) {
            if (tile + 2 * (int)gridDim.x < ntiles) issue(order(tile + 2 * gridDim.x), cur, &bar[s]);
            if constexpr (C::TSTORE) {
                // store the previous tile: every thread wrote and fenced its
                // part of the output buffer before the barrier above
                if (it > 0) {
                    const S *o = s ? out0 : out1;
#pragma unroll
                    for (int i = 0; i < 9; i++) tma_store_3d(&tdst, o + i * OPE, px0, py0, i);
                    bulk_commit();
                }
            }
        }
#pragma unroll
        for (int j = 0; j < C::NQ; j++) {
            const int ly = ly0 + j * DY;
            F2 dxr(0.f), dyr(0.f);
            if constexpr (DRHO) pair_gradients<C::RW>(Rs + (ly + 1) * C::RW + x + 2, kf.inv12, kf.inv12r, dxr, dyr);
            F2 ux, uy, drho;
            if constexpr (!C::TSTORE) collide_moments<F2, FORCE>(k, g[j], mom[j]);
            collide_relax<F2, DRHO, FORCE>(k, mom[j], g[j], dxr, dyr, ux, uy, drho);
            const long long o = (long long)(y0 + ly) * gd.pitch + (x0 + x);
            if constexpr (C::TSTORE) {
                S *ob = (s ? out1 : out0) + ly * W + x;
#pragma unroll
                for (int i = 0; i < 9; i++) Pair<S>::store(ob + i * OPE, g[j][i]);
            } else {
#pragma unroll
                for (int i = 0; i < 9; i++) Pair<S>::store(dst + (long long)i * gd.plane + o, g[j][i]);
            }
            if constexpr (EPI) {
                if (own_x & (y0 + ly >= oy)) {
                    __stcs(reinterpret_cast<float2 *>(snap + o), ux.v);
                    const float da = ux.v.x - snv[j].x, db = ux.v.y - snv[j].y;
                    acc.add(da * da, drho.v.x);
                    acc.add(db * db, drho.v.y);
                }
            }
        }
        if constexpr (C::TSTORE) fence_async_shared();  // this thread's output-tile writes, before the next barrier
        px0 = x0;
        py0 = y0;
    }
    __syncthreads();  // every collision is done: R is free
    if constexpr (C::TSTORE) {
        if (tid == PROD && it > 0) {  // the last tile's store
            const S *o = ((it - 1) & 1) ? out1 : out0;
#pragma unroll
            for (int i = 0; i < 9; i++) tma_store_3d(&tdst, o + i * OPE, px0, py0, i);
            bulk_commit();
        }
    }
    // edge strips: general tile body, density tile in R
    for (int e = blockIdx.x; e < edge.start[edge.n]; e += gridDim.x) {
        int ex0, ey0, ex1, ey1, lw;
        rect_tile(edge, e, ex0, ey0, ex1, ey1, lw);
        general_tile<S, float, DRHO, EPI, FORCE>(src, dst, gd, kf, snap, ex0, ey0, ex1, ey1, lw, acc, R);
    }
    if constexpr (EPI) {
        __shared__ double red[2 * (THREADS / 32)];
        double a, b;
        acc.block_total(a, b, red);
        if (tid == 0) partials[blockIdx.x] = make_double2(a, b);
    }
    if constexpr (C::TSTORE) {
        if (tid == PROD) bulk_wait_all();  // the output tiles stay allocated until the stores are done
    }
}

}  // namespace prc
