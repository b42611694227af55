// prc_batch_tma.cuh -- the batch engine with TMA-staged interior tiles.
//
// Same contract as k_batch (prc_batch.cuh): one cooperative persistent launch
// advances every active instance by up to `steps` time steps, a bounded grid
// barrier per step, per-instance bookkeeping and retirement.  The tiles differ:
//   * the interior of each instance (nodes at least two from every wall) is
//     covered by 64 x 8 tiles whose source windows -- the tile plus a one-node
//     ring, shifted by -e_i, one per population plane -- come into shared
//     memory by nine tiled TMA copies through the instance's own descriptors,
//     two tiles in flight per CTA, exactly as in the single-instance interior
//     kernel k_step_tma (one node pair per thread, the same pulls, density
//     ring, gradients and packed FP32x2 collision, so an instance's
//     populations are bitwise those of a single handle on that kernel);
//   * the edge strips use the general tile body with L2-coherent loads, and
//     a grid too small for one interior tile is covered by the general
//     kernel's 64 x 8 node-pair tiles (as a single handle on variant 0 does).
// The CTAs take the global tile list strided by the grid size; in each, one
// producer thread walks its tiles two ahead, skips the tiles of retired
// instances, stages each tile's windows and its instance's coefficients, and
// hands the tile to the CTA through a record in shared memory that the
// tile's barrier publishes.  Used when every instance of the launch
// has the density-gradient terms, no body force and the central-moment
// scheme, FP32 or FP16 storage.
#pragma once

#include "prc_batch.cuh"

namespace prc {

constexpr int BT_W = 64, BT_H = 8, BT_THREADS = 256;

template <typename S>
using BatchTmaCfg = TmaCfg<S, BT_W, BT_H, BT_THREADS>;

// Order this thread's later async-proxy (TMA) reads of global memory after
// the generic-proxy writes it has synchronised with (the previous step's
// stores by every CTA, made visible by the grid barrier).
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// A staged interior tile: global tile index (-1: none), instance, step count
// of the instance, tile origin (x0, y0) and nominal origin (ox, oy; the last
// row / column of tiles is shifted back, see Interior).
struct BatchTile {
    int q, i;
    long long t;
    int x0, y0, ox, oy;
};

// What the tile walk needs of an instance, copied into shared memory at the
// start of every step (with the CTA's one decision on whether the instance
// is active in that step), so that the producer never waits on global
// memory for it.
struct BatchTileInst {
    const CUtensorMap *tmap;
    long long t;  // the instance's step count in this step
    int itile_start, ntx, xlast, ylast;
    int slot, active;
    int etile_start;
};

constexpr int BT_MAX_INST = 512;  // instances of a launch of k_batch_tma at most
// Coefficient buffers, used in turn by consecutive tiles: the copy for the
// tile after next lands while this tile's collision still reads its buffer,
// and the buffer of the tile before, free since this tile's barrier, is the
// one it overwrites (three would do; four index cheaply).
constexpr int BT_CBUF = 4;

template <typename S>
__host__ __device__ constexpr int batch_tma_smem()
{
    using C = BatchTmaCfg<S>;
    // stages, density tiles, coefficient buffers, instance table, barriers, base alignment
    return 2 * C::STAGE_BYTES + 2 * C::R_BYTES + BT_CBUF * (int)sizeof(BatchCoef<float>) +
           BT_MAX_INST * (int)sizeof(BatchTileInst) + 128 + 128;
}

// Bring a tensor-map descriptor (in global memory) into the TMA unit's cache
// ahead of the copies that use it.
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

template <typename S>
__global__ void __launch_bounds__(BT_THREADS, 2)
k_batch_tma(const BatchInst *__restrict__ inst, const BatchCoef<float> *__restrict__ coefs, BatchDyn *dyn, int ninst,
            int total_itiles, int total_etiles, double2 *partials, BatchCtl *ctl, int steps)
{
    using C = BatchTmaCfg<S>;
    constexpr int W = C::W, H = C::H;
    static_assert(C::NQ == 1, "one node pair per thread");
    constexpr int PE = C::PLANE_BYTES / (int)sizeof(S);  // plane stride in elements
    constexpr int RF = C::R_BYTES / (int)sizeof(float);  // floats per density tile
    constexpr int RING = 2 * C::PAIRS + 2 * C::RH;        // ring units
    constexpr int CB = (int)sizeof(BatchCoef<float>);
    static_assert(RING <= BT_THREADS - 32, "one ring unit per thread at most, none in the producer's warp");
    static_assert(C::R_BYTES >= srho_floats(BT_THREADS) * (int)sizeof(float), "density tile too small for the strips");
    static_assert(C::R_BYTES >= PAIR_SRHO * (int)sizeof(float), "density tile too small for the pair tiles");
    static_assert(CB % 16 == 0 && C::STAGE_BYTES % 128 == 0 && C::R_BYTES % 128 == 0, "16-byte bulk copies");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    S *stage0 = reinterpret_cast<S *>(smem);
    S *stage1 = reinterpret_cast<S *>(smem + C::STAGE_BYTES);
    float *R = reinterpret_cast<float *>(smem + 2 * C::STAGE_BYTES);
    BatchCoef<float> *cstage = reinterpret_cast<BatchCoef<float> *>(smem + 2 * C::STAGE_BYTES + 2 * C::R_BYTES);
    BatchTileInst *tinst =
        reinterpret_cast<BatchTileInst *>(smem + 2 * C::STAGE_BYTES + 2 * C::R_BYTES + BT_CBUF * CB);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * C::STAGE_BYTES + 2 * C::R_BYTES + BT_CBUF * CB +
                                                 BT_MAX_INST * (int)sizeof(BatchTileInst));
    __shared__ BatchTile rec[2];
    __shared__ double red[2 * (BT_THREADS / 32)];

    const int tid = threadIdx.x;
    const int ly = tid / C::PAIRS, x = 2 * (tid - ly * C::PAIRS);  // this thread's pair in a tile
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t ph = 0;  // bit b: parity of the next completion of bar[b]

    // The CTA's interior tiles are the global list strided by the grid size,
    // so that neighbouring tiles are staged at about the same time by
    // neighbouring CTAs and their shared window rows and columns come from
    // L2.  The producer thread (lane 0 of the last warp, which has no ring
    // work and would otherwise wait at the tile barrier) walks them: it finds
    // the next tile before the barrier and, right after it, issues the tile's
    // nine window copies into the freed stage and one bulk copy of its
    // instance's coefficients, both completing on the stage's barrier.
    const bool producer = tid == BT_THREADS - 32;
    int nq = 0, wi = 0;
    auto pick = [&]() {
        BatchTile r;
        r.q = -1;
        while (nq < total_itiles) {
            while (wi + 1 < ninst && nq >= tinst[wi + 1].itile_start) wi++;  // tiles are in instance order
            const BatchTileInst &e = tinst[wi];
            const int q = nq;
            nq += gridDim.x;
            if (!e.active) continue;
            const int lt = q - e.itile_start;
            const int ty = lt / e.ntx;
            r.q = q;
            r.i = wi;
            r.t = e.t;
            r.ox = C::PADX + (lt - ty * e.ntx) * W;  // interior origin (PADX, 2), see make_batch_tma_plan
            r.oy = 2 + ty * H;
            r.x0 = min(r.ox, e.xlast);
            r.y0 = min(r.oy, e.ylast);
            break;
        }
        return r;
    };
    auto issue = [&](int st, const BatchTile &r, int cb) {
        rec[st] = r;
        if (r.q >= 0) {
            const BatchTileInst &e = tinst[r.i];
            S *stg = st ? stage1 : stage0;
            const CUtensorMap *map = e.tmap + (int)(r.t & 1);
            mbar_arrive_expect_tx(&bar[st], 9u * C::BOX_BYTES + CB);
#pragma unroll
            for (int i = 0; i < 9; i++) tma_load_3d(stg + i * PE, map, &bar[st], r.x0 - C::PADX, r.y0 - 1 - ey_of(i), i);
            bulk_load(cstage + cb, coefs + e.slot, CB, &bar[st]);
        }
    };

    for (int s = 0; s < steps; s++) {
        // ---- the instance table of this step: one activity decision per
        // instance for the whole CTA (the state may change meanwhile)
        for (int k = tid; k < ninst; k += BT_THREADS) {
            const BatchInst &I = inst[k];
            BatchTileInst e;
            e.tmap = I.tmap;
            e.t = I.t0 + s;
            e.itile_start = I.itile_start;
            e.ntx = I.in.ntx;
            e.xlast = I.in.xlast;
            e.ylast = I.in.ylast;
            e.slot = I.slot;
            e.active = ld_relaxed_i32(&dyn[I.slot].state) == BATCH_ACTIVE && e.t < I.max_steps;
            e.etile_start = I.etile_start;
            tinst[k] = e;
        }
        __syncthreads();
        // ---- interior tiles, TMA-staged
        // producer: the tile after the two in flight, picked one tile early so
        // that its descriptor is prefetched by the time its copies are issued
        BatchTile nxt;
        if (producer) {
            fence_proxy_async_global();
            nq = blockIdx.x;
            wi = 0;
            issue(0, pick(), 0);
            issue(1, pick(), 1);
            nxt = pick();
            if (nxt.q >= 0) prefetch_tmap(tinst[nxt.i].tmap + (int)(nxt.t & 1));
        }
        __syncthreads();  // the first two records
        for (int it = 0;; it++) {
            const int st = it & 1;
            // this tile's record: the producer rewrites it after the tile's
            // barrier, and the rewrite becomes visible at the next tile's barrier
            const BatchTile r = rec[st];
            if (r.q < 0) break;  // no later record holds a tile either
            // read now, used after the collision: the loads overlap the wait and the pulls
            const BatchInst &I = inst[r.i];
            const bool epi = ((r.t + 1) % 20) == 0;
            const bool own = (r.x0 + x >= r.ox) & (r.y0 + ly >= r.oy);
            float *snap = static_cast<float *>(I.snap);
            S *dst = static_cast<S *>(I.pop[(int)(r.t & 1) ^ 1]);
            const long long plane = I.gd.plane;
            const long long o = (long long)(r.y0 + ly) * I.gd.pitch + (r.x0 + x);
            float2 snv = make_float2(0.f, 0.f);
            if (epi && own) snv = __ldcs(reinterpret_cast<const float2 *>(snap + o));
            const S *cur = st ? stage1 : stage0;
            float *Rs = R + st * RF;
            // a thread whose wait runs out still pulls (stale shared memory) so
            // that every thread reaches the barrier, which takes the vote
            const bool ok = mbar_wait_bounded(&bar[st], (ph >> st) & 1u);
            ph ^= 1u << st;
            F2 g[9];
            pull_pair<S, PE>(cur + (ly + 1) * C::BW + x + C::PADX, g);
            *reinterpret_cast<float2 *>(Rs + (ly + 1) * C::RW + x + 2) = sum9(g).v;
            if (tid < RING) ring_density<S, W, H, PE, C::BW, C::RW, C::PADX>(tid, cur, Rs);
            BatchTile nn;  // producer: the tile after nxt
            if (producer) {
                nn = pick();
                if (nn.q >= 0) prefetch_tmap(tinst[nn.i].tmap + (int)(nn.t & 1));
            }
            if (__syncthreads_or(!ok)) {
                if (producer) {
                    atomicExch(&ctl->error, 1);
                    // the copies of the next tile may be outstanding
                    if (rec[st ^ 1].q >= 0) mbar_wait_bounded(&bar[st ^ 1], (ph >> (st ^ 1)) & 1u);
                }
                return;
            }
            // the coefficients staged with this tile (buffer it mod BT_CBUF)
            const BatchCoef<float> &K = cstage[it & (BT_CBUF - 1)];
            if (producer) {  // every pull from this stage is done
                issue(st, nxt, (it + 2) & (BT_CBUF - 1));
                nxt = nn;
            }
            F2 dxr, dyr;
            pair_gradients<C::RW>(Rs + (ly + 1) * C::RW + x + 2, K.k.inv12, K.k.inv12r, dxr, dyr);
            F2 ux, uy, drho;
            collide<F2, true, false>(K.k2, g, dxr, dyr, ux, uy, drho);
#pragma unroll
            for (int i = 0; i < 9; i++) Pair<S>::store(dst + (long long)i * plane + o, g[i]);
            if (epi) {  // uniform across the CTA: one instance per tile
                RedAcc<float> acc;
                if (own) {
                    __stcs(reinterpret_cast<float2 *>(snap + o), ux.v);
                    const float da = ux.v.x - snv.x, db = ux.v.y - snv.y;
                    acc.add(da * da, drho.v.x);
                    acc.add(db * db, drho.v.y);
                }
                double a, b;
                acc.block_total(a, b, red);
                if (tid == 0) partials[I.part_base + (r.q - I.itile_start)] = make_double2(a, b);
                __syncthreads();  // red is reused by the next total
            }
        }
        // ---- edge strips: general tile body, L2-coherent loads, density tile
        // in R; the CTA's edge tiles strided over the global edge-tile list
        // (their instances found in the shared table, not in global memory)
        {
            int ei = 0;
            for (int e = blockIdx.x; e < total_etiles; e += gridDim.x) {
                while (ei + 1 < ninst && e >= tinst[ei + 1].etile_start) ei++;
                if (!tinst[ei].active) continue;
                const BatchInst &I = inst[ei];
                const long long t = tinst[ei].t;
                const int le = e - I.etile_start;
                const S *src = static_cast<const S *>(I.pop[(int)(t & 1)]);
                S *dst = static_cast<S *>(I.pop[(int)(t & 1) ^ 1]);
                float *snap = static_cast<float *>(I.snap);
                const BatchCoef<float> &K = coefs[I.slot];
                const bool epi = ((t + 1) % 20) == 0;
                RedAcc<float> acc;
                if (I.in.ntx == 0) {
                    // a grid without interior tiles: the 64 x 8 node-pair tiles of
                    // the general kernel (what a single handle runs on it)
                    const int x0 = (le % I.tiles_x) * PTW, y0 = (le / I.tiles_x) * PTH;
                    if (epi) pair_tile<S, true, true, false, true, false>(src, dst, I.gd, K.k, K.k2, snap, x0, y0, acc, R);
                    else pair_tile<S, true, false, false, true, false>(src, dst, I.gd, K.k, K.k2, snap, x0, y0, acc, R);
                } else {
                    int ex0, ey0, ex1, ey1, lw;
                    rect_tile(I.edge, le, ex0, ey0, ex1, ey1, lw);
                    if (epi)
                        general_tile<S, float, true, true, false, true>(src, dst, I.gd, K.k, snap, ex0, ey0, ex1, ey1,
                                                                        lw, acc, R);
                    else
                        general_tile<S, float, true, false, false, true>(src, dst, I.gd, K.k, snap, ex0, ey0, ex1, ey1,
                                                                         lw, acc, R);
                }
                if (epi) {
                    double a, b;
                    acc.block_total(a, b, red);
                    if (tid == 0) partials[I.part_base + I.in.ntx * I.in.nty + le] = make_double2(a, b);
                    __syncthreads();  // red is reused by the next total
                }
            }
        }
        if (!grid_barrier(ctl)) return;
        batch_bookkeeping(inst, dyn, ninst, partials, tid);
        // As in k_batch, no second barrier: the next step's tiles may start
        // while this bookkeeping runs (the tiles take the step count from t0).
    }
}

}  // namespace prc
