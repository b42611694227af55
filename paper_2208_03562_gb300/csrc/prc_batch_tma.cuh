// prc_batch_tma.cuh -- the batch engine with TMA-staged tiles.
//
// Same contract as k_batch (prc_batch.cuh): one cooperative persistent launch
// advances every active instance by up to `steps` time steps, a bounded grid
// barrier per step, per-instance bookkeeping and retirement.  The tiles differ:
// each instance is covered by 64 x 8 node tiles at origins (64 tx, 8 ty), the
// last column and row reaching past the grid, and every tile's source windows
// -- one per population plane, shifted by -e_i -- come into shared memory by
// nine tiled TMA copies through the instance's own descriptors, two tiles in
// flight per CTA, one node pair per thread.
//   * A tile whose nodes and one-node density ring all lie at least one node
//     inside the walls (an interior tile) runs the single-instance interior
//     kernel's tile body (k_step_tma): windows of the tile plus the ring, the
//     same pulls, density ring, gradients and packed FP32x2 collision.
//   * Any other tile (a wall tile) takes windows two rows taller (one more
//     row below and above), which hold, for every node of the tile and of its
//     ring, both its pulls and all nine of its own populations.  One pass
//     copies, for each node at a wall, its own opposite populations into the
//     out-of-grid window cells that its pulls across the wall read (ghost
//     cells), so that the plain pulls stream with half-way bounce-back; the
//     moving-lid term is added to the two diagonal links of the top row
//     (reading A3).  The density gradient reads its eight neighbours at
//     positions clamped into the grid (the nearest fluid node's density
//     beyond a wall, reading A1); only nodes inside the grid are stored.
// Every node computes what the general tile body computes for it (the same
// pulls, density sums, stencil and collision, in the same order), so an
// instance's populations are bitwise those of a single handle on the 64 x 8
// interior-kernel variant, whose edge strips take the general tile body.
// The CTAs take the global tile list strided by the grid size for about 7/8
// of it and claim the rest from a counter; in each, one
// producer thread walks its tiles two ahead, skips the tiles of retired
// instances, stages each tile's windows and its instance's coefficients, and
// hands the tile to the CTA through a record in shared memory that the tile's
// barrier publishes.  Used when every instance of the launch is a cavity with
// the density-gradient terms, no body force and the central-moment scheme,
// FP32 or FP16 storage.
#pragma once

#include "prc_batch.cuh"

namespace prc {

constexpr int BT_W = 64, BT_H = 8, BT_THREADS = 256;
static_assert(BT_W == PTW && BT_H == BY, "the batch tiles of both bodies share one tiling and one partial-sum layout");

template <typename S>
struct BatchTmaCfg {
    static constexpr int W = BT_W, H = BT_H;
    static constexpr int PADX = 16 / (int)sizeof(S);  // 16-byte aligned box start
    static constexpr int BW = W + 2 * PADX;           // box width (elements)
    static constexpr int BH = H + 2;                  // interior tiles: tile + ring rows
    static constexpr int BHW = H + 4;                 // wall tiles: one more row below and above
    static constexpr int BOX_BYTES = BW * BH * (int)sizeof(S);
    static constexpr int BOXW_BYTES = BW * BHW * (int)sizeof(S);
    static constexpr int PLANE_BYTES = (BOXW_BYTES + 127) / 128 * 128;  // one plane slot holds either box
    static constexpr int STAGE_BYTES = 9 * PLANE_BYTES;
    static constexpr int RW = W + 4, RH = H + 2;  // density tile: node lx of row ly at (ly + 1) RW + lx + 2
    static constexpr int R_BYTES = (RW * RH * 4 + 127) / 128 * 128;
    static constexpr int PAIRS = W / 2;
};

// Order this thread's later async-proxy (TMA) reads of global memory after
// the generic-proxy writes it has synchronised with (the previous step's
// stores by every CTA, made visible by the grid barrier).
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// A staged tile: global tile index (-1: none), instance, origin, whether it
// is a wall tile, the parity of the instance's step count (its source set)
// and whether the step is one of the instance's residual steps.
struct BatchTile {
    int q, i;
    int x0, y0, wall;
    int par, epi;
};

// What the tile walk needs of an instance, copied into shared memory at the
// start of every step (with the CTA's one decision on whether the instance
// is active in that step), so that the producer never waits on global
// memory for it.
struct BatchTileInst {
    const CUtensorMap *tmap;  // [interior box: set 0, set 1; wall box: set 0, set 1]
    int tile_start, ntx, nx, ny;
    int slot, active, lid_on;
    int par, epi;  // the instance's step count in this step: parity, and whether it ends a residual interval
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

// ---- wall tiles.  `cw` is the stage one row into the taller windows, so
// that a node of tile row ly pulls from window row ly + 1 and a node of ring
// row ry (0: below the tile, H + 1: above it) from row ry, as in the interior
// body; a node at absolute row y sits in the window of plane p at row
// y - y0 + 1 + e_py (relative to cw).

// Ghost cells of a wall tile (half-way bounce-back, reading A3): for every
// node n of the tile or its ring that lies inside the grid and every
// population i whose source n - e_i lies beyond a wall, the window of plane i
// at n - e_i -- a position outside the grid, which the copy filled with zeros
// and which no other pull reads -- receives the node's own population
// opp(i), so that the plain pulls then stream with bounce-back.  The cells of
// one wall are those of its nodes (one column or row of the tile and ring)
// and of the three populations that point away from it; a corner cell is
// written twice with the same value.  The moving-lid term is added after
// the pull, in the collision precision (lid_pull).  All threads take part;
// the caller synchronises before the pulls.
template <typename S, int W, int H, int PE, int BW, int PADX, int THREADS>
__device__ __forceinline__ void fill_ghosts(S *cw, int tid, int x0, int y0, int nx, int ny)
{
    constexpr int NV = (H + 2) * 3, NH = (W + 2) * 3;  // cells of a vertical / horizontal wall
    const bool wl = x0 == 0, wr = (nx - 1 >= x0 - 1) & (nx - 1 <= x0 + W);
    const bool wb = y0 == 0, wt = (ny - 1 >= y0 - 1) & (ny - 1 <= y0 + H);
    const int total = (wl ? NV : 0) + (wr ? NV : 0) + (wb ? NH : 0) + (wt ? NH : 0);
    bool wrote = false;
    for (int c = tid; c < total; c += THREADS) {
        int k = c, side;  // 0 left, 1 right, 2 bottom, 3 top
        const int n0 = wl ? NV : 0, n1 = wr ? NV : 0, n2 = wb ? NH : 0;
        if (k < n0) {
            side = 0;
        } else if ((k -= n0) < n1) {
            side = 1;
        } else if ((k -= n1) < n2) {
            side = 2;
        } else {
            k -= n2;
            side = 3;
        }
        const int sel = k % 3, along = k / 3;
        int ax, ay, i;
        if (side < 2) {
            ax = side == 0 ? 0 : nx - 1;
            ay = y0 - 1 + along;
            i = side == 0 ? (sel == 0 ? 1 : (sel == 1 ? 5 : 8)) : (sel == 0 ? 3 : (sel == 1 ? 6 : 7));
        } else {
            ax = x0 - 1 + along;
            ay = side == 2 ? 0 : ny - 1;
            i = side == 2 ? (sel == 0 ? 2 : (sel == 1 ? 5 : 6)) : (sel == 0 ? 4 : (sel == 1 ? 7 : 8));
        }
        if ((ax < 0) | (ax >= nx) | (ay < 0) | (ay >= ny)) continue;
        // e_i and the opposite direction, for i in 1..8 (Eq. 3 ordering)
        const int exi = (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
        const int eyi = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
        const int j = i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5;
        const int col = ax - x0 + PADX, row = ay - y0 + 1;
        cw[i * PE + row * BW + col - exi] = cw[j * PE + (row - eyi) * BW + col];
        wrote = true;
    }
    // the next copies into this stage (async proxy) come after these writes
    if (wrote) fence_async_shared();
}

// The moving-lid term of the pulls from above the top wall (the two
// diagonal links SW and SE of a node in the top row, reading A3), added to
// the bounced populations in the collision precision as pull9 does.
template <typename V>
__device__ __forceinline__ void lid_pull(V g[9], float lid);
template <>
__device__ __forceinline__ void lid_pull<float>(float g[9], float lid)
{
    g[7] -= lid;
    g[8] += lid;
}
template <>
__device__ __forceinline__ void lid_pull<F2>(F2 g[9], float lid)
{
    g[7].v.x -= lid;
    g[7].v.y -= lid;
    g[8].v.x += lid;
    g[8].v.y += lid;
}

// Density of one ring unit of a wall tile (the units of ring_density) from
// the ghost-filled windows, with the lid term for a unit in the top row.
// Units outside the grid form values that the clamped gradients never read.
template <typename S, int W, int H, int PE, int BW, int RW, int PADX>
__device__ __forceinline__ void ring_density_wall(int tid, const S *cw, float *Rs, int y0, int ny, bool lid_on,
                                                  float lid)
{
    constexpr int PAIRS = W / 2;
    if (tid < 2 * PAIRS) {
        const int ry = tid < PAIRS ? 0 : H + 1;
        const int rx = 2 * (tid < PAIRS ? tid : tid - PAIRS);
        F2 gr[9];
        pull_pair<S, PE>(cw + ry * BW + rx + PADX, gr);
        if (lid_on & (y0 - 1 + ry == ny - 1)) lid_pull(gr, lid);
        *reinterpret_cast<float2 *>(Rs + ry * RW + rx + 2) = sum9(gr).v;
    } else {
        const int c = tid - 2 * PAIRS;
        const int ry = c >> 1, lx = (c & 1) ? W : -1;
        const S *b = cw + ry * BW + lx + PADX;
        float gr[9];
#pragma unroll
        for (int i = 0; i < 9; i++) gr[i] = Pair<S>::one(b + i * PE - ex_of(i));
        if (lid_on & (y0 - 1 + ry == ny - 1)) lid_pull(gr, lid);
        Rs[ry * RW + lx + 2] = sum9(gr);
    }
}

// Density gradients (reading A1) of the node (ax, ay) at tile position
// (lx, ly), its neighbours' positions clamped into the grid (the stencil and
// operation order of general_tile).
template <int RW>
__device__ __forceinline__ void node_gradients_clamped(const float *Rs, int lx, int ly, int ax, int ay, int nx, int ny,
                                                       float i12, float i12r, float &dxr, float &dyr)
{
    const int xc = lx + 2, xw = (ax > 0 ? lx - 1 : lx) + 2, xe = (ax + 1 < nx ? lx + 1 : lx) + 2;
    const int yc = (ly + 1) * RW, ys = (ay > 0 ? ly : ly + 1) * RW, yn = (ay + 1 < ny ? ly + 2 : ly + 1) * RW;
    const float rE = Rs[yc + xe], rW = Rs[yc + xw];
    const float rN = Rs[yn + xc], rS = Rs[ys + xc];
    const float rNE = Rs[yn + xe], rNW = Rs[yn + xw];
    const float rSE = Rs[ys + xe], rSW = Rs[ys + xw];
    drho_stencil<float>(rE, rW, rN, rS, rNE, rNW, rSE, rSW, i12, i12r, dxr, dyr);
}

template <typename S>
struct Scalar;
template <>
struct Scalar<float> {
    static __device__ __forceinline__ void store(float *p, float v) { *p = v; }
};
template <>
struct Scalar<__half> {
    static __device__ __forceinline__ void store(__half *p, float v) { *p = __float2half_rn(v); }
};

template <typename S>
__global__ void __launch_bounds__(BT_THREADS, 2)
k_batch_tma(const BatchInst *__restrict__ inst, const BatchCoef<float> *__restrict__ coefs, BatchDyn *dyn, int ninst,
            int total_tiles, double2 *partials, BatchCtl *ctl, int steps)
{
    using C = BatchTmaCfg<S>;
    constexpr int W = C::W, H = C::H;
    static_assert(H * C::PAIRS == BT_THREADS, "one node pair per thread");
    constexpr int PE = C::PLANE_BYTES / (int)sizeof(S);  // plane stride in elements
    constexpr int RF = C::R_BYTES / (int)sizeof(float);  // floats per density tile
    constexpr int RING = 2 * C::PAIRS + 2 * C::RH;        // ring units
    constexpr int CB = (int)sizeof(BatchCoef<float>);
    static_assert(RING <= BT_THREADS - 32, "one ring unit per thread at most, none in the producer's warp");
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

    // Tile assignment.  A CTA first takes its tiles statically, strided by the
    // grid size (blockIdx.x, + grid, + 2 grid, ...: neighbouring tiles are
    // staged at about the same time by neighbouring CTAs, and their shared
    // window rows and columns come from L2), NS of them, about 7/8 of an
    // equal share; the remaining tiles, from NS grid on, are claimed one at a
    // time from a launch-wide counter, so that a CTA that ran ahead takes
    // more of them.  With fixed equal shares the CTAs of a large launch
    // waited at each step's grid barrier for 8-14 % of the time; claiming
    // every tile measured slower than this split (an atomic per tile), and
    // claiming the last quarter no better.  Claim numbers of step s start at
    // s (D + grid), D = max(0, tiles - NS grid): each CTA makes exactly one
    // claim past the end (the one that ends its step), so a step takes
    // D + grid claims.  One claim is always in flight: the next is requested
    // as soon as the previous is taken, a tile ahead of its use.  The producer
    // thread (lane 0 of the last warp, which has no ring work and would
    // otherwise wait at the tile barrier) walks the tiles: it finds the next
    // tile before the barrier and, right after it, issues the tile's nine
    // window copies into the freed stage and one bulk copy of its instance's
    // coefficients, both completing on the stage's barrier.
    const bool producer = tid == BT_THREADS - 32;
    const int G = gridDim.x;
    const int NS = max(3, total_tiles / G - max(2, total_tiles / (8 * G)));
    const long long dyn_tiles = total_tiles > NS * G ? (long long)total_tiles - (long long)NS * G : 0;
    int wi = 0, nstatic = 0;
    bool ended = false;
    unsigned long long kp = 0;  // the claim in flight
    long long base = 0;         // first claim number of this step
    auto pick = [&]() {
        BatchTile r;
        r.q = -1;
        for (;;) {
            long long q;
            if (nstatic < NS) {
                q = blockIdx.x + (long long)nstatic * G;
                nstatic = q < total_tiles ? nstatic + 1 : NS;
                if (q >= total_tiles) continue;
            } else {
                if (ended) break;
                q = (long long)NS * G + ((long long)kp - base);
                if (q >= total_tiles) {
                    ended = true;
                    break;
                }
                kp = atomicAdd(&ctl->claim, 1ULL);
            }
            while (wi + 1 < ninst && q >= tinst[wi + 1].tile_start) wi++;  // tiles are in instance order
            const BatchTileInst &e = tinst[wi];
            if (!e.active) continue;
            const int lt = (int)q - e.tile_start;
            const int ty = lt / e.ntx;
            r.q = (int)q;
            r.i = wi;
            r.par = e.par;
            r.epi = e.epi;
            r.x0 = (lt - ty * e.ntx) * W;
            r.y0 = ty * H;
            // interior: every node of the tile and of its ring at least one
            // node inside the walls (their pulls need no bounce-back)
            r.wall = !((r.x0 >= 2) & (r.x0 + W + 2 <= e.nx) & (r.y0 >= 2) & (r.y0 + H + 2 <= e.ny));
            break;
        }
        return r;
    };
    auto tmap_of = [&](const BatchTile &r) { return tinst[r.i].tmap + 2 * r.wall + r.par; };
    auto issue = [&](int st, const BatchTile &r, int cb) {
        rec[st] = r;
        if (r.q >= 0) {
            const BatchTileInst &e = tinst[r.i];
            S *stg = st ? stage1 : stage0;
            const CUtensorMap *map = tmap_of(r);
            mbar_arrive_expect_tx(&bar[st], 9u * (r.wall ? C::BOXW_BYTES : C::BOX_BYTES) + CB);
            const int yb = r.y0 - 1 - r.wall;  // first window row for e_y = 0
#pragma unroll
            for (int i = 0; i < 9; i++) tma_load_3d(stg + i * PE, map, &bar[st], r.x0 - C::PADX, yb - ey_of(i), i);
            bulk_load(cstage + cb, coefs + e.slot, CB, &bar[st]);
        }
    };

    for (int s = 0; s < steps; s++) {
        // ---- the instance table of this step: one activity decision per
        // instance for the whole CTA (the state may change meanwhile)
        for (int k = tid; k < ninst; k += BT_THREADS) {
            const BatchInst &I = inst[k];
            BatchTileInst e;
            const long long t = I.t0 + s;
            e.tmap = I.tmap;
            e.par = (int)(t & 1);
            e.epi = (t + 1) % 20 == 0;
            e.tile_start = I.tile_start;
            e.ntx = I.tiles_x;
            e.nx = I.gd.nx;
            e.ny = I.gd.ny;
            e.slot = I.slot;
            e.active = ld_relaxed_i32(&dyn[I.slot].state) == BATCH_ACTIVE && t < I.max_steps;
            e.lid_on = I.gd.lid_on;
            tinst[k] = e;
        }
        __syncthreads();
        // producer: the tile after the two in flight, picked one tile early so
        // that its descriptor is prefetched by the time its copies are issued
        BatchTile nxt;
        if (producer) {
            fence_proxy_async_global();
            base = (long long)s * (dyn_tiles + G);
            kp = atomicAdd(&ctl->claim, 1ULL);  // taken after the static tiles
            nstatic = 0;
            ended = false;
            wi = 0;
            issue(0, pick(), 0);
            issue(1, pick(), 1);
            nxt = pick();
            if (nxt.q >= 0) prefetch_tmap(tmap_of(nxt));
        }
        __syncthreads();  // the first two records
        for (int it = 0;; it++) {
            const int st = it & 1;
            // this tile's record: the producer rewrites it after the tile's
            // barrier, and the rewrite becomes visible at the next tile's barrier
            const BatchTile r = rec[st];
            if (r.q < 0) break;  // no later record holds a tile either
            const BatchTileInst &e = tinst[r.i];
            // read now, used after the collision: the loads overlap the wait and the pulls
            const BatchInst &I = inst[r.i];
            const bool epi = r.epi != 0;
            const int nx = e.nx, ny = e.ny;
            const int ax = r.x0 + x, ay = r.y0 + ly;  // this thread's first node
            const bool v0 = (ax < nx) & (ay < ny), v1 = (ax + 1 < nx) & (ay < ny);
            float *snap = static_cast<float *>(I.snap);
            S *dst = static_cast<S *>(I.pop[r.par ^ 1]);
            const long long plane = I.gd.plane;
            const long long o = (long long)ay * I.gd.pitch + ax;
            float2 snv = make_float2(0.f, 0.f);
            if (epi) {
                if (v1) snv = __ldcs(reinterpret_cast<const float2 *>(snap + o));
                else if (v0) snv.x = __ldcs(snap + o);
            }
            const S *cur = st ? stage1 : stage0;
            float *Rs = R + st * RF;
            // the coefficients staged with this tile (buffer it mod BT_CBUF)
            const BatchCoef<float> &K = cstage[it & (BT_CBUF - 1)];
            // a thread whose wait runs out still pulls (stale shared memory) so
            // that every thread reaches the barrier, which takes the vote
            const bool ok = mbar_wait_bounded(&bar[st], (ph >> st) & 1u);
            ph ^= 1u << st;
            F2 g[9];
            if (!r.wall) {  // uniform across the CTA: one tile per CTA at a time
                pull_pair<S, PE>(cur + (ly + 1) * C::BW + x + C::PADX, g);
                *reinterpret_cast<float2 *>(Rs + (ly + 1) * C::RW + x + 2) = sum9(g).v;
                if (tid < RING) ring_density<S, W, H, PE, C::BW, C::RW, C::PADX>(tid, cur, Rs);
            } else {
                S *cw = (st ? stage1 : stage0) + C::BW;
                const bool lid_on = e.lid_on != 0;
                fill_ghosts<S, W, H, PE, C::BW, C::PADX, BT_THREADS>(cw, tid, r.x0, r.y0, nx, ny);
                __syncthreads();  // every ghost cell of the stage is written
                pull_pair<S, PE>(cw + (ly + 1) * C::BW + x + C::PADX, g);
                if (lid_on & (ay == ny - 1)) lid_pull(g, K.k.lid);
                *reinterpret_cast<float2 *>(Rs + (ly + 1) * C::RW + x + 2) = sum9(g).v;
                if (tid < RING)
                    ring_density_wall<S, W, H, PE, C::BW, C::RW, C::PADX>(tid, cw, Rs, r.y0, ny, lid_on, K.k.lid);
            }
            BatchTile nn;  // producer: the tile after nxt
            if (producer) {
                nn = pick();
                if (nn.q >= 0) prefetch_tmap(tmap_of(nn));
            }
            if (__syncthreads_or(!ok)) {
                if (producer) {
                    atomicExch(&ctl->error, 1);
                    // the copies of the next tile may be outstanding
                    if (rec[st ^ 1].q >= 0) mbar_wait_bounded(&bar[st ^ 1], (ph >> (st ^ 1)) & 1u);
                }
                return;
            }
            if (producer) {  // every pull from this stage is done
                issue(st, nxt, (it + 2) & (BT_CBUF - 1));
                nxt = nn;
            }
            F2 dxr, dyr;
            if (!r.wall || ((ax >= 1) & (ax + 2 < nx) & (ay >= 1) & (ay + 1 < ny))) {
                pair_gradients<C::RW>(Rs + (ly + 1) * C::RW + x + 2, K.k.inv12, K.k.inv12r, dxr, dyr);
            } else {
                dxr = F2(0.f);
                dyr = F2(0.f);
                if (v0) node_gradients_clamped<C::RW>(Rs, x, ly, ax, ay, nx, ny, K.k.inv12, K.k.inv12r, dxr.v.x, dyr.v.x);
                if (v1)
                    node_gradients_clamped<C::RW>(Rs, x + 1, ly, ax + 1, ay, nx, ny, K.k.inv12, K.k.inv12r, dxr.v.y,
                                                  dyr.v.y);
            }
            F2 ux, uy, drho;
            collide<F2, true, false>(K.k2, g, dxr, dyr, ux, uy, drho);
            if (v1) {
#pragma unroll
                for (int i = 0; i < 9; i++) Pair<S>::store(dst + (long long)i * plane + o, g[i]);
            } else if (v0) {
#pragma unroll
                for (int i = 0; i < 9; i++) Scalar<S>::store(dst + (long long)i * plane + o, g[i].v.x);
            }
            if (epi) {  // uniform across the CTA: one instance per tile
                RedAcc<float> acc;
                if (v1) {
                    __stcs(reinterpret_cast<float2 *>(snap + o), ux.v);
                    const float da = ux.v.x - snv.x, db = ux.v.y - snv.y;
                    acc.add(da * da, drho.v.x);
                    acc.add(db * db, drho.v.y);
                } else if (v0) {
                    __stcs(snap + o, ux.v.x);
                    const float da = ux.v.x - snv.x;
                    acc.add(da * da, drho.v.x);
                }
                double a, b;
                acc.block_total(a, b, red);
                if (tid == 0) partials[I.part_base + (r.q - I.tile_start)] = make_double2(a, b);
                __syncthreads();  // red is reused by the next total
            }
        }
        if (!grid_barrier(ctl)) return;
        batch_bookkeeping(inst, dyn, ninst, partials, tid);
        // As in k_batch, no second barrier: the next step's tiles may start
        // while this bookkeeping runs (the tiles take the step count from t0).
    }
}

}  // namespace prc
