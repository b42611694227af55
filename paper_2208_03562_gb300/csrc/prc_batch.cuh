// prc_batch.cuh -- many independent cavities in one persistent launch.
//
// A batch is a table of instances, each with its own grid, parameters,
// population sets, residual snapshot and step counter.  One cooperative launch
// of k_batch advances every active instance by up to `steps` time steps: in
// each step the CTAs sweep the tiles of all active instances (wall-aware tile
// body: 64 x 8 nodes in pairs for the FP32 collision, 32 x 8 for FP64), a grid barrier separates the steps, and after each
// residual step (every 20 steps of an instance's own counter) one CTA per
// instance reduces that instance's per-tile partial sums in a fixed order,
// so an instance's result does not depend on the other instances of the mix.
// An instance retires when its residual falls below its tolerance, when it
// diverges, when it reaches its step limit, or (optional) when its residual
// stalls: at the first residual evaluation at least `stall_window` steps after
// the previous checkpoint, a residual above stall_ratio times the checkpoint's
// retires the instance as STALLED (a precision floor: the rounding noise of the
// storage format keeps the residual from falling further).  Its result is the
// set of the step at which it retired; its tiles are skipped from the next
// step on, or from the one after (the next step's tiles may start before the
// bookkeeping that retires it ends; see k_batch), and that one extra step
// writes only the other set.  One grid barrier per step separates the tiles
// from the bookkeeping; it is a bounded spin: when it runs out it records
// LBM_ETIMEOUT and every CTA leaves.
#pragma once

#include <type_traits>

#include "prc_pair.cuh"
#include "prc_tma.cuh"

namespace prc {

// Per-slot coefficient table entry: the collision constants in the collision
// type and, for the FP32 collision, packed for the pair tile body.
// 16-byte aligned and sized, so that one bulk copy can bring a slot's entry
// into shared memory.
template <typename T>
struct alignas(16) BatchCoef {
    Coef<T> k;
    Coef<F2> k2;
};

// Tile of the batch engine: 64 x 8 nodes (pair tile body) for the FP32
// collision, 32 x 8 (one node per thread) for FP64.
template <typename T>
__host__ __device__ constexpr int batch_tile_w() { return std::is_same<T, float>::value ? PTW : BX; }

enum BatchState : int {
    BATCH_ACTIVE = 0,
    BATCH_CONVERGED = 1,
    BATCH_DIVERGED = 2,
    BATCH_MAXSTEPS = 3,
    BATCH_EMPTY = 4,
    BATCH_STALLED = 5
};

// Read-only part of an instance descriptor (set by the host before a launch).
struct BatchInst {
    int slot;           // index into the per-slot tables (coefficients, dynamic state)
    int pad;
    void *pop[2];       // population sets A / B (state in pop[t & 1])
    void *snap;         // residual snapshot (u_x), collision precision
    Grid gd;
    int tiles_x, tiles;  // BX x BY tiling of the grid
    int tile_start;      // first global tile index of this instance in the launch
    int part_base;       // first partial-sum slot
    long long t0;        // completed steps at the start of the launch
    int drho, force;
    double tol;
    long long max_steps;
    long long stall_window;  // steps between stall checkpoints (0: no stall test)
    double stall_ratio;      // stalled when res > stall_ratio * checkpoint residual
    // TMA-staged tile body (k_batch_tma): the same tiles, staged through the
    // slot's load descriptors in device memory, interior box (tile + ring) of
    // pop[0] and pop[1], then wall box (two rows taller) of both
    const CUtensorMap *tmap;
};

// Mutable part, updated on the device.
struct BatchDyn {
    long long t;         // completed steps
    long long res_step;  // step of the last residual
    double res, mass;
    int state;
    int pad;
    long long chk_step;  // stall checkpoint: step and residual
    double chk_res;
};

struct BatchCtl {
    unsigned arrive;     // grid barrier
    unsigned gen;
    int error;           // 1: barrier timeout
    int hold;            // failure-detection check: CTA 0 withholds its first arrival
    long long limit;     // wait limit of the grid barrier in SM clock cycles (0: about two seconds)
    unsigned long long claim;  // tile claims of k_batch_tma, counted over the launch
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid barrier for a cooperative (co-resident) launch; false when it
// timed out or another CTA reported an error.
__device__ __forceinline__ bool grid_barrier(BatchCtl *ctl)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        ok = 1;
        const unsigned g = ld_acquire_u32(&ctl->gen);
        __threadfence();
        const unsigned n = gridDim.x;
        const long long limit = ctl->limit > 0 ? ctl->limit : 4000000000LL;  // about two seconds by default
        // (check of the failure detection) CTA 0 withholds its arrival, so
        // that every other CTA's wait runs out; it then waits out its own
        if (ctl->hold && blockIdx.x == 0) {
            const long long t0 = clock64();
            while (ld_acquire_u32(&ctl->gen) == g && !ld_relaxed_i32(&ctl->error) && clock64() - t0 <= limit)
                __nanosleep(64);
            atomicExch(&ctl->error, 1);
            ok = 0;
        } else if (atomicAdd(&ctl->arrive, 1u) == n - 1) {
            atomicExch(&ctl->arrive, 0u);
            __threadfence();
            atomicAdd(&ctl->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire_u32(&ctl->gen) == g) {
                if (ld_relaxed_i32(&ctl->error)) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > limit) {
                    atomicExch(&ctl->error, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Shared memory of k_batch: the density tile of a tile (+ ring), declared once
// for every instantiation of the tile body.
template <typename S, typename T>
__host__ __device__ constexpr int batch_smem_bytes()
{
    return std::is_same<T, float>::value ? PAIR_SRHO * 4 : srho_floats(BX * BY) * (int)sizeof(T);
}

template <typename S, typename T, bool DRHO, bool EPI, bool FORCE, bool RAW>
__device__ __forceinline__ void batch_tile_t(const BatchInst &I, const BatchCoef<T> &k, int parity, int lt,
                                             double2 *partials, unsigned char *bsm)
{
    RedAcc<T> acc;
    if constexpr (std::is_same<T, float>::value) {
        float *srho = reinterpret_cast<float *>(bsm);
        const int x0 = (lt % I.tiles_x) * PTW, y0 = (lt / I.tiles_x) * PTH;
        pair_tile<S, DRHO, EPI, FORCE, true, RAW>(static_cast<const S *>(I.pop[parity]),
                                                 static_cast<S *>(I.pop[parity ^ 1]), I.gd, k.k, k.k2,
                                                 static_cast<float *>(I.snap), x0, y0, acc, srho);
    } else {
        T *srho = reinterpret_cast<T *>(bsm);
        const int x0 = (lt % I.tiles_x) * BX, y0 = (lt / I.tiles_x) * BY;
        general_tile<S, T, DRHO, EPI, FORCE, true, RAW>(static_cast<const S *>(I.pop[parity]),
                                                   static_cast<S *>(I.pop[parity ^ 1]), I.gd, k.k,
                                                   static_cast<T *>(I.snap), x0, y0, I.gd.nx, I.gd.ny, 5, acc,
                                                   srho);
    }
    if constexpr (EPI) {
        __shared__ double red[2 * (BX * BY / 32)];
        double a, b;
        acc.block_total(a, b, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[I.part_base + lt] = make_double2(a, b);
        __syncthreads();  // red may be reused by the next tile of this CTA
    }
}

template <typename S, typename T, bool RAW>
__device__ __forceinline__ void batch_tile_m(const BatchInst &I, const BatchCoef<T> &k, int parity, int lt, bool epi,
                                             double2 *partials, unsigned char *bsm)
{
    if (I.drho) {
        if (I.force) {
            if (epi) batch_tile_t<S, T, true, true, true, RAW>(I, k, parity, lt, partials, bsm);
            else batch_tile_t<S, T, true, false, true, RAW>(I, k, parity, lt, partials, bsm);
        } else {
            if (epi) batch_tile_t<S, T, true, true, false, RAW>(I, k, parity, lt, partials, bsm);
            else batch_tile_t<S, T, true, false, false, RAW>(I, k, parity, lt, partials, bsm);
        }
    } else {
        if (I.force) {
            if (epi) batch_tile_t<S, T, false, true, true, RAW>(I, k, parity, lt, partials, bsm);
            else batch_tile_t<S, T, false, false, true, RAW>(I, k, parity, lt, partials, bsm);
        } else {
            if (epi) batch_tile_t<S, T, false, true, false, RAW>(I, k, parity, lt, partials, bsm);
            else batch_tile_t<S, T, false, false, false, RAW>(I, k, parity, lt, partials, bsm);
        }
    }
}

template <typename S, typename T>
__device__ __forceinline__ void batch_tile(const BatchInst &I, const BatchCoef<T> &k, int parity, int lt, bool epi,
                                           double2 *partials, unsigned char *bsm)
{
    if (I.gd.model == 1) batch_tile_m<S, T, true>(I, k, parity, lt, epi, partials, bsm);
    else batch_tile_m<S, T, false>(I, k, parity, lt, epi, partials, bsm);
}

// Bookkeeping after the tiles of one step: counters, residuals, retirement
// (one CTA per instance).  Thread 0 reads the instance's state and counter
// once into shared memory and is the only writer; the barriers keep every
// branch below uniform across the CTA (a thread that re-read D->t after
// thread 0 advanced it would take a different branch).  CTAs of 256 threads.
__device__ __forceinline__ void batch_bookkeeping(const BatchInst *__restrict__ inst, BatchDyn *dyn, int ninst,
                                                  const double2 *partials, int tid)
{
    constexpr int NT = BX * BY;
    __shared__ long long sh_t;
    __shared__ int sh_active;
    for (int j = blockIdx.x; j < ninst; j += gridDim.x) {
        const BatchInst &I = inst[j];
        BatchDyn *D = dyn + I.slot;
        __syncthreads();  // the previous instance's shared values are consumed
        if (tid == 0) {
            sh_active = ld_relaxed_i32(&D->state) == BATCH_ACTIVE;
            sh_t = __ldcg(&D->t) + 1;
        }
        __syncthreads();
        if (!sh_active) continue;
        const long long t = sh_t;
        if (t % 20 == 0) {
            __shared__ double sa[NT], sb[NT];
            double a = 0.0, b = 0.0;
            for (int q = tid; q < I.tiles; q += NT) {
                const double2 v = __ldcg(partials + I.part_base + q);
                a += v.x;
                b += v.y;
            }
            sa[tid] = a;
            sb[tid] = b;
            __syncthreads();
            for (int w = NT / 2; w > 0; w >>= 1) {
                if (tid < w) {
                    sa[tid] += sa[tid + w];
                    sb[tid] += sb[tid + w];
                }
                __syncthreads();
            }
            if (tid == 0) {
                const double res = sqrt(sa[0]), mass = (double)I.gd.nx * (double)I.gd.ny + sb[0];
                D->res = res;
                D->mass = mass;
                D->res_step = t;
                if (!isfinite(res) || !isfinite(mass)) D->state = BATCH_DIVERGED;
                else if (res < I.tol) D->state = BATCH_CONVERGED;
                else if (I.stall_window > 0 && t - D->chk_step >= I.stall_window) {
                    if (D->chk_step > 0 && res > I.stall_ratio * D->chk_res) D->state = BATCH_STALLED;
                    D->chk_step = t;
                    D->chk_res = res;
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            D->t = t;
            if (D->state == BATCH_ACTIVE && t >= I.max_steps) D->state = BATCH_MAXSTEPS;
        }
    }
}

// SPEC = 1: every instance of the launch has the density-gradient terms on,
// no body force and the central-moment scheme, so the tile body is chosen at
// compile time (a smaller kernel); SPEC = 0 dispatches per instance.
template <typename S, typename T, int SPEC>
__global__ void __launch_bounds__(BX * BY, 3)
k_batch(const BatchInst *__restrict__ inst, const BatchCoef<T> *__restrict__ coefs, BatchDyn *dyn, int ninst,
        int total_tiles, double2 *partials, BatchCtl *ctl, int steps)
{
    const int tid = threadIdx.y * BX + threadIdx.x;
    __shared__ __align__(16) unsigned char bsm[batch_smem_bytes<S, T>()];
    for (int s = 0; s < steps; s++) {
        // ---- one time step of every active instance
        int i = 0;
        int ci = -1;         // instance whose state and counter were read last (they change only between steps)
        bool active = false, epi = false;
        long long t = 0;
        for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
            while (i + 1 < ninst && tile >= inst[i + 1].tile_start) i++;  // tiles are in instance order
            const BatchInst &I = inst[i];
            if (i != ci) {
                ci = i;
                // an active instance has completed t0 + s steps; its state may
                // be changing right now (see the bookkeeping below), so the
                // CTA takes one decision for all its threads
                t = I.t0 + s;
                active = __syncthreads_and(ld_relaxed_i32(&dyn[I.slot].state) == BATCH_ACTIVE && t < I.max_steps);
                epi = ((t + 1) % 20) == 0;
            }
            if (!active) continue;
            if constexpr (SPEC == 1) {
                if (epi) batch_tile_t<S, T, true, true, false, false>(I, coefs[I.slot], (int)(t & 1), tile - I.tile_start,
                                                                   partials, bsm);
                else batch_tile_t<S, T, true, false, false, false>(I, coefs[I.slot], (int)(t & 1), tile - I.tile_start,
                                                                  partials, bsm);
            } else {
                batch_tile<S, T>(I, coefs[I.slot], (int)(t & 1), tile - I.tile_start, epi, partials, bsm);
            }
        }
        if (!grid_barrier(ctl)) return;
        batch_bookkeeping(inst, dyn, ninst, partials, tid);
        // No grid barrier here: the next step's tiles start while the
        // bookkeeping of this one may still run.  Each instance's bookkeeping
        // is done by one CTA, which alone writes its counter and state; the
        // tiles take the step count from t0.  A tile that reads the state just
        // before the instance is retired advances it once more: retirement by
        // the residual (converged, diverged, stalled) happens at a residual
        // step, so that extra step is not one (no snapshot or partial-sum
        // writes), and it reads the instance's final set and writes only the
        // other one.  The step limit is checked in the tiles themselves.  The
        // partial sums that this bookkeeping reads are written again only 20
        // steps later.
    }
}

}  // namespace prc
