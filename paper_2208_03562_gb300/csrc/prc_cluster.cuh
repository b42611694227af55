// prc_cluster.cuh -- cluster-resident engine for small grids.
//
// One thread-block cluster holds a whole instance in distributed shared
// memory for many time steps.  CTA c of the cluster owns the rows
// [c rpc, min((c + 1) rpc, ny)) ("slab"), both population sets of its slab
// and a density tile of the slab plus a one-node ring.  One time step:
//   1. density tile: rho - rho0 of every slab node and of the ring, each from
//      its nine pulled populations (App. A streaming; reading A1 for ghost
//      nodes); pulls of rows outside the slab read the neighbouring CTA's
//      shared memory through the cluster's distributed shared memory;
//   2. CTA barrier;
//   3. every slab node: pull, density gradient from the tile, collision
//      (the same `collide` as every other kernel, on pairs of neighbouring
//      nodes in packed FP32x2 arithmetic for the FP32 collision, as in the
//      general kernel, so the populations are bitwise those of the general
//      kernel), store into the other set;
//   4. cluster barrier: the new set is complete before anyone pulls from it.
// Every 20th step of the absolute step counter the CTAs add their FP64
// residual / mass totals in rank order (identically in every CTA, so the
// stop decision is uniform and no CTA waits on a barrier the others skip).
// The state is read from global memory at launch and written back at the end,
// so a launch of n steps costs one global read and write of the state instead
// of n; steps are separated by cluster barriers instead of kernel launches.
#pragma once

#include <cooperative_groups.h>

#include <type_traits>

#include "prc_kernels.cuh"

namespace prc {

constexpr int CL_THREADS = 512;
constexpr int CL_MAX_CTAS = 16;

struct ClusterGeom {
    int nc;    // CTAs (slabs)
    int rpc;   // rows per slab (the last may be shorter, never below 2)
    int smem;  // dynamic shared memory per CTA (bytes)
};

// Shared-memory footprint of a slab of `rows` rows, nx wide.
__host__ __device__ inline size_t cluster_smem_bytes(int rows, int nx, size_t elem, size_t telem)
{
    const size_t f = 2 * 9 * (size_t)rows * nx * elem;
    const size_t fa = (f + 15) / 16 * 16;
    return fa + (size_t)(rows + 2) * (nx + 2) * telem;
}

// Load of one stored population through a 32-bit shared::cluster address
// (this CTA's shared memory or another CTA's of the cluster), widened to the
// collision type.  Volatile: the loads must stay between the cluster
// barriers that order them against the neighbours' stores.
template <typename S, typename T>
__device__ __forceinline__ T ld_cl(uint32_t a);
template <>
__device__ __forceinline__ double ld_cl<double, double>(uint32_t a)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
template <>
__device__ __forceinline__ float ld_cl<float, float>(uint32_t a)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
template <>
__device__ __forceinline__ float ld_cl<__half, float>(uint32_t a)
{
    unsigned short v;
    asm volatile("ld.shared::cluster.b16 %0, [%1];" : "=h"(v) : "r"(a));
    return __half2float(__ushort_as_half(v));
}

// The two halves of a cluster barrier: arrive (releasing this thread's
// earlier writes) and wait for every CTA's arrival (acquiring theirs).  Work
// that needs none of the other CTAs' data can run between them.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// shared::cta address of a pointer into this CTA's shared memory
__device__ __forceinline__ uint32_t cta_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// the same location in the shared memory of CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(uint32_t cta_addr, int rank)
{
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(cta_addr), "r"(rank));
    return a;
}

// Read access to one population set of the cluster in 32-bit shared::cluster
// addresses: this CTA's slab, the two neighbouring slabs (rows within two of
// the slab) and, across a periodic wrap, any slab.  Every CTA lays its set
// out the same way: plane i, local row ly, column x at i plane_b + ly row_b +
// x sizeof(S) from the set's base.
struct SlabView {
    uint32_t own, prev, next;  // base of the set in this CTA and in the neighbouring CTAs
    uint32_t own_cta;          // base of the set in this CTA's shared::cta window (mapa source on a wrap)
    int y_lo, y_hi, rpc, nc;
    uint32_t row_b, plane_b;   // bytes per row and per plane

    // address of plane 0, column 0 of the in-domain row y (any slab)
    __device__ __forceinline__ uint32_t row(int y) const
    {
        if (y >= y_lo && y < y_hi) return own + (uint32_t)(y - y_lo) * row_b;
        if (y < y_lo && y >= y_lo - 2) return prev + (uint32_t)(y - (y_lo - rpc)) * row_b;
        if (y >= y_hi && y < y_hi + 2) return next + (uint32_t)(y - y_hi) * row_b;
        const int owner = min(y / rpc, nc - 1);  // periodic wrap across the first / last slab
        return cluster_addr(own_cta, owner) + (uint32_t)(y - owner * rpc) * row_b;
    }
};

// Pull-streaming with half-way bounce-back and the lid (as pull9) through
// the slab view.  Nodes whose nine sources are all inside the domain (away
// from the x walls, and away from the y walls unless y is periodic) take the
// fast path: the three source rows are resolved once and the nine pulls are
// fixed offsets from them.
template <typename S, typename T>
__device__ __forceinline__ void pull9_slab(const SlabView &v, const Grid &gd, int x, int y, T lid, T g[9])
{
    constexpr uint32_t es = sizeof(S);
    const bool xin = (x >= 1) & (x <= gd.nx - 2);
    const bool yin = (gd.bc == 2) | ((y >= 1) & (y <= gd.ny - 2));
    if (xin & yin) {
        const int ym = y == 0 ? gd.ny - 1 : y - 1, yp = y == gd.ny - 1 ? 0 : y + 1;
        const uint32_t rr[3] = {v.row(ym), v.row(y), v.row(yp)};  // source row of e_y = +1, 0, -1
#pragma unroll
        for (int i = 0; i < 9; i++)
            g[i] = ld_cl<S, T>(rr[1 - ey_of(i)] + (uint32_t)i * v.plane_b + (uint32_t)(x - ex_of(i)) * es);
        return;
    }
    const uint32_t here = v.row(y) + (uint32_t)x * es;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        int sx = x - ex_of(i), sy = y - ey_of(i);
        if (gd.bc >= 1) sx = sx < 0 ? sx + gd.nx : (sx >= gd.nx ? sx - gd.nx : sx);
        if (gd.bc == 2) sy = sy < 0 ? sy + gd.ny : (sy >= gd.ny ? sy - gd.ny : sy);
        const bool inside = (sx >= 0) & (sx < gd.nx) & (sy >= 0) & (sy < gd.ny);
        if (inside) {
            g[i] = ld_cl<S, T>(v.row(sy) + (uint32_t)i * v.plane_b + (uint32_t)sx * es);
        } else {
            T w = ld_cl<S, T>(here + (uint32_t)opp_of(i) * v.plane_b);
            if (sy >= gd.ny && gd.lid_on) {
                if (i == 7) w -= lid;
                if (i == 8) w += lid;
            }
            g[i] = w;
        }
    }
}

// The nine pulls of the node pair (x, x + 1) in FP32, one pair of source rows
// resolved for both nodes when all eighteen sources are inside the domain.
template <typename S>
__device__ __forceinline__ void pull_pair_slab(const SlabView &v, const Grid &gd, int x, int y, bool v1,
                                               float lid, float ga[9], float gb[9])
{
    constexpr uint32_t es = sizeof(S);
    const bool fast = (x >= 1) & (x + 2 <= gd.nx - 1) & ((gd.bc == 2) | ((y >= 1) & (y <= gd.ny - 2)));
    if (fast) {
        const int ym = y == 0 ? gd.ny - 1 : y - 1, yp = y == gd.ny - 1 ? 0 : y + 1;
        const uint32_t rr[3] = {v.row(ym), v.row(y), v.row(yp)};
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const uint32_t a = rr[1 - ey_of(i)] + (uint32_t)i * v.plane_b + (uint32_t)(x - ex_of(i)) * es;
            ga[i] = ld_cl<S, float>(a);
            gb[i] = ld_cl<S, float>(a + es);
        }
        return;
    }
    pull9_slab<S, float>(v, gd, x, y, lid, ga);
    if (v1) pull9_slab<S, float>(v, gd, x + 1, y, lid, gb);
    else
#pragma unroll
        for (int i = 0; i < 9; i++) gb[i] = ga[i];
}

// n time steps of one instance on one cluster (gridDim.x == cluster size).
// pop_in holds the state after step t0; the state after the last step done
// goes to pop_out[parity of that step].
// ONE (FP32 collision only): every slab holds at most one node pair per
// thread, and only that path is compiled into the kernel.
template <typename S, typename T, bool DRHO, bool FORCE, bool RAW, bool ONE>
__global__ void __launch_bounds__(CL_THREADS, 1)
k_cluster(const S *__restrict__ pop0, const S *__restrict__ pop1, Grid gd, Coef<T> k, Coef<F2> k2,
          T *__restrict__ snap, DevStatus *__restrict__ st, long long t0, int nsteps, int rpc)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char cl_smem[];
    __shared__ double2 part;      // this CTA's residual / mass totals
    __shared__ double red[2 * (CL_THREADS / 32)];
    __shared__ int sh_stop;

    if (st->stop) return;  // uniform: read before any write by this launch
    const int nc = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int nx = gd.nx;
    const int plane = rpc * nx;  // elements per plane of a slab (the same layout in every CTA)
    SlabView v;
    v.rpc = rpc;
    v.nc = nc;
    v.y_lo = rank * rpc;
    v.y_hi = min(v.y_lo + rpc, gd.ny);
    v.row_b = (uint32_t)nx * (uint32_t)sizeof(S);
    v.plane_b = (uint32_t)plane * (uint32_t)sizeof(S);
    const int rows = v.y_hi - v.y_lo;
    const size_t fbytes = (2 * 9 * (size_t)rpc * nx * sizeof(S) + 15) / 16 * 16;
    S *F0 = reinterpret_cast<S *>(cl_smem);
    S *F1 = F0 + 9 * plane;
    T *rho = reinterpret_cast<T *>(cl_smem + fbytes);
    const int prv = rank > 0 ? rank - 1 : nc - 1, nxt = rank + 1 < nc ? rank + 1 : 0;
    // 32-bit shared::cluster addresses of both sets in this CTA and its neighbours
    const uint32_t own0c = cta_smem_addr(F0), own1c = cta_smem_addr(F1);  // shared::cta window
    const uint32_t own0 = cluster_addr(own0c, rank), own1 = cluster_addr(own1c, rank);
    const uint32_t prev0 = cluster_addr(own0c, prv), prev1 = cluster_addr(own1c, prv);
    const uint32_t next0 = cluster_addr(own0c, nxt), next1 = cluster_addr(own1c, nxt);

    // load the slab of the current state
    const S *pin = (t0 & 1) ? pop1 : pop0;
    const int nslab = rows * nx;
    // this thread's nodes q = tid + k nthr of the slab (ly = q / nx, x = q % nx)
    // and of the density tile (q / RW, q % RW), advanced without divisions
    const int RW = nx + 2;
    const int s_dly = nthr / nx, s_dx = nthr - s_dly * nx;
    const int s_ly0 = tid / nx, s_x0 = tid - s_ly0 * nx;
    const int r_dly = nthr / RW, r_dx = nthr - r_dly * RW;
    const int r_ly0 = tid / RW, r_x0 = tid - r_ly0 * RW;
    for (int i = 0; i < 9; i++)
        for (int q = tid; q < nslab; q += nthr) {
            const int ly = q / nx, x = q - ly * nx;
            F0[i * plane + ly * nx + x] =
                pin[(long long)i * gd.plane + (long long)(v.y_lo + ly) * gd.pitch + x];
        }
    __syncthreads();
    cluster_arrive();  // matched by the wait at the top of the first step

    // One pair per thread (FP32 collision, slabs of at most `nthr` pairs):
    // this thread's pair and its ring node are the same every step, so the
    // addresses of their source rows in both sets are resolved once here and
    // the per-step pulls are fixed offsets from them.
    constexpr uint32_t es = sizeof(S);
    const int npx1 = (nx + 1) >> 1;
    const int p_ly = tid / npx1, p_x = 2 * (tid - p_ly * npx1), p_y = v.y_lo + p_ly;
    const bool p_fast = (tid < rows * npx1) & (p_x >= 1) & (p_x + 2 <= nx - 1) &
                        ((gd.bc == 2) | ((p_y >= 1) & (p_y <= gd.ny - 2)));
    const int nring1 = 2 * RW + 2 * rows;  // density-tile ring: rows -1 and `rows`, columns -1 and nx
    int r_lx = 0, r_rl = 0, r_gx = 0, r_gy = 0;
    if (tid < nring1) {
        if (tid < RW) {
            r_lx = tid - 1;
            r_rl = -1;
        } else if (tid < 2 * RW) {
            r_lx = tid - RW - 1;
            r_rl = rows;
        } else if (tid < 2 * RW + rows) {
            r_lx = -1;
            r_rl = tid - 2 * RW;
        } else {
            r_lx = nx;
            r_rl = tid - 2 * RW - rows;
        }
        r_gx = r_lx;
        r_gy = v.y_lo + r_rl;
        map_node(gd, r_gx, r_gy);
    }
    const bool r_fast = (tid < nring1) & (r_gx >= 1) & (r_gx <= nx - 2) &
                        ((gd.bc == 2) | ((r_gy >= 1) & (r_gy <= gd.ny - 2)));
    uint32_t pr0[3] = {0, 0, 0}, pr1[3] = {0, 0, 0}, rr0[3] = {0, 0, 0}, rr1[3] = {0, 0, 0};
    if constexpr (ONE)
    for (int sb = 0; sb < 2; sb++) {
        v.own = sb ? own1 : own0;
        v.own_cta = sb ? own1c : own0c;
        v.prev = sb ? prev1 : prev0;
        v.next = sb ? next1 : next0;
        uint32_t *pr = sb ? pr1 : pr0, *rr = sb ? rr1 : rr0;
        if (p_fast) {
            const int ym = p_y == 0 ? gd.ny - 1 : p_y - 1, yp = p_y == gd.ny - 1 ? 0 : p_y + 1;
            pr[0] = v.row(ym) + (uint32_t)p_x * es;  // source row of e_y = +1, 0, -1, at column p_x
            pr[1] = v.row(p_y) + (uint32_t)p_x * es;
            pr[2] = v.row(yp) + (uint32_t)p_x * es;
        }
        if (r_fast) {
            const int ym = r_gy == 0 ? gd.ny - 1 : r_gy - 1, yp = r_gy == gd.ny - 1 ? 0 : r_gy + 1;
            rr[0] = v.row(ym) + (uint32_t)r_gx * es;
            rr[1] = v.row(r_gy) + (uint32_t)r_gx * es;
            rr[2] = v.row(yp) + (uint32_t)r_gx * es;
        }
    }

    int b = 0;  // set holding the state
    int done = 0;
    bool waited = false;  // the last cluster barrier phase has been waited on
    const double nnodes = (double)gd.nx * (double)gd.ny;
    int t20 = (int)((t0 + 1) % 20);  // index of the step being made, modulo 20
    for (; done < nsteps; done++, t20 = t20 == 19 ? 0 : t20 + 1) {
        const long long t = t0 + done + 1;  // absolute index of the step being made
        const bool epi = t20 == 0;
        v.own = b ? own1 : own0;
        v.own_cta = b ? own1c : own0c;
        v.prev = b ? prev1 : prev0;
        v.next = b ? next1 : next0;
        S *Fo = b ? F0 : F1;
        // 1. density tile (slab + ring), one node at a time
        auto density_pass = [&]() {
            const int nr = (rows + 2) * RW;
            int ry = r_ly0, rx = r_x0;
            for (int q = tid; q < nr; q += nthr) {
                const int ly = ry - 1, lx = rx - 1;
                rx += r_dx;
                ry += r_dly;
                if (rx >= RW) {
                    rx -= RW;
                    ry++;
                }
                int gx = lx, gy = v.y_lo + ly;
                map_node(gd, gx, gy);
                T g[9];
                pull9_slab<S, T>(v, gd, gx, gy, k.lid, g);
                rho[q] = sum9(g);
            }
            __syncthreads();
        };
        RedAcc<T> acc;
        if constexpr (std::is_same<T, float>::value) {
            // FP32 collision: pairs of neighbouring nodes (x, x + 1), x even,
            // in packed FP32x2 arithmetic, as in the general kernel
            const int npx = (nx + 1) >> 1, npairs = rows * npx;
            // 2. collide one pair (pulled values in ga, gb) into the other set
            auto pair_body = [&](int ly, int x, const float *ga, const float *gb) {
                const int y = v.y_lo + ly;
                const bool v1 = x + 1 < nx;
                F2 g[9];
#pragma unroll
                for (int i = 0; i < 9; i++) g[i] = F2(ga[i], gb[i]);
                float dx[2] = {0.f, 0.f}, dy[2] = {0.f, 0.f};
                if constexpr (DRHO) {
#pragma unroll
                    for (int j = 0; j < 2; j++) {
                        const float *c = rho + (ly + 1) * RW + x + j + 1;
                        const float rE = c[1], rW = c[-1];
                        const float rN = c[RW], rS = c[-RW];
                        const float rNE = c[RW + 1], rNW = c[RW - 1];
                        const float rSE = c[-RW + 1], rSW = c[-RW - 1];
                        drho_stencil<float>(rE, rW, rN, rS, rNE, rNW, rSE, rSW, k.inv12, k.inv12r, dx[j], dy[j]);
                    }
                }
                F2 ux, uy, drho;
                collide<F2, DRHO, FORCE, RAW>(k2, g, F2(dx[0], dx[1]), F2(dy[0], dy[1]), ux, uy, drho);
                const int o = ly * nx + x;
#pragma unroll
                for (int i = 0; i < 9; i++) {
                    Fo[i * plane + o] = to_s<S, float>(g[i].v.x);
                    if (v1) Fo[i * plane + o + 1] = to_s<S, float>(g[i].v.y);
                }
                if (epi) {
                    const long long og = (long long)y * gd.pitch + x;
                    const float d0 = ux.v.x - snap[og];
                    snap[og] = ux.v.x;
                    acc.add(d0 * d0, drho.v.x);
                    if (v1) {
                        const float d1 = ux.v.y - snap[og + 1];
                        snap[og + 1] = ux.v.y;
                        acc.add(d1 * d1, drho.v.y);
                    }
                }
            };
            if constexpr (ONE) {
                // one pair per thread: its pulls stay in registers across the
                // density barrier, and the density pass only adds the ring
                const bool act = tid < npairs;
                const int ly = p_ly, x = p_x;
                float ga[9], gb[9];
                auto fast_pulls = [&]() {
                    const uint32_t r0 = b ? pr1[0] : pr0[0], r1 = b ? pr1[1] : pr0[1], r2 = b ? pr1[2] : pr0[2];
#pragma unroll
                    for (int i = 0; i < 9; i++) {
                        const uint32_t a = (ey_of(i) == 1 ? r0 : (ey_of(i) == 0 ? r1 : r2)) + (uint32_t)i * v.plane_b -
                                           (uint32_t)(ex_of(i) * (int)es);
                        ga[i] = ld_cl<S, float>(a);
                        gb[i] = ld_cl<S, float>(a + es);
                    }
                };
                // a pair whose source rows all lie in this CTA's slab pulls
                // before waiting for the other CTAs of the previous step
                const bool early = p_fast & (ly >= 1) & (ly <= rows - 2);
                if (early) fast_pulls();
                cluster_wait();
                if (early) {
                } else if (p_fast) {
                    fast_pulls();
                } else if (act) {
                    pull_pair_slab<S>(v, gd, x, v.y_lo + ly, x + 1 < nx, k.lid, ga, gb);
                }
                if constexpr (DRHO) {
                    if (act) {
                        rho[(ly + 1) * RW + x + 1] = sum9(ga);
                        if (x + 1 < nx) rho[(ly + 1) * RW + x + 2] = sum9(gb);
                    }
                    if (r_fast) {  // this thread's ring node, sources inside the domain
                        const uint32_t r0 = b ? rr1[0] : rr0[0], r1 = b ? rr1[1] : rr0[1], r2 = b ? rr1[2] : rr0[2];
                        float gr[9];
#pragma unroll
                        for (int i = 0; i < 9; i++)
                            gr[i] = ld_cl<S, float>((ey_of(i) == 1 ? r0 : (ey_of(i) == 0 ? r1 : r2)) +
                                                    (uint32_t)i * v.plane_b - (uint32_t)(ex_of(i) * (int)es));
                        rho[(r_rl + 1) * RW + r_lx + 1] = sum9(gr);
                    }
                    const int nring = nring1;
                    for (int q = r_fast ? tid + nthr : tid; q < nring; q += nthr) {
                        int lx, rl;
                        if (q < RW) {
                            lx = q - 1;
                            rl = -1;
                        } else if (q < 2 * RW) {
                            lx = q - RW - 1;
                            rl = rows;
                        } else if (q < 2 * RW + rows) {
                            lx = -1;
                            rl = q - 2 * RW;
                        } else {
                            lx = nx;
                            rl = q - 2 * RW - rows;
                        }
                        int gx = lx, gy = v.y_lo + rl;
                        map_node(gd, gx, gy);
                        float gr[9];
                        pull9_slab<S, float>(v, gd, gx, gy, k.lid, gr);
                        rho[(rl + 1) * RW + lx + 1] = sum9(gr);
                    }
                    __syncthreads();
                }
                if (act) pair_body(ly, x, ga, gb);
            } else {
                cluster_wait();
                if constexpr (DRHO) density_pass();
                const int p_dly = nthr / npx, p_dx = nthr - p_dly * npx;
                int py = tid / npx, pxi = tid - py * npx;
                for (int q = tid; q < npairs; q += nthr) {
                    const int ly = py, x = 2 * pxi;
                    pxi += p_dx;
                    py += p_dly;
                    if (pxi >= npx) {
                        pxi -= npx;
                        py++;
                    }
                    float ga[9], gb[9];
                    pull_pair_slab<S>(v, gd, x, v.y_lo + ly, x + 1 < nx, k.lid, ga, gb);
                    pair_body(ly, x, ga, gb);
                }
            }
        } else {
            // FP64 collision: one node at a time
            cluster_wait();
            if constexpr (DRHO) density_pass();
            int sy_ = s_ly0, sx_ = s_x0;
            for (int q = tid; q < nslab; q += nthr) {
                const int ly = sy_, x = sx_;
                sx_ += s_dx;
                sy_ += s_dly;
                if (sx_ >= nx) {
                    sx_ -= nx;
                    sy_++;
                }
                const int y = v.y_lo + ly;
                T g[9];
                pull9_slab<S, T>(v, gd, x, y, k.lid, g);
                T dxr = T(0), dyr = T(0);
                if constexpr (DRHO) {
                    const T *c = rho + (ly + 1) * RW + x + 1;
                    const T rE = c[1], rW = c[-1];
                    const T rN = c[RW], rS = c[-RW];
                    const T rNE = c[RW + 1], rNW = c[RW - 1];
                    const T rSE = c[-RW + 1], rSW = c[-RW - 1];
                    drho_stencil<T>(rE, rW, rN, rS, rNE, rNW, rSE, rSW, k.inv12, k.inv12r, dxr, dyr);
                }
                T ux, uy, drho;
                collide<T, DRHO, FORCE, RAW>(k, g, dxr, dyr, ux, uy, drho);
                const int o = ly * nx + x;
#pragma unroll
                for (int i = 0; i < 9; i++) Fo[i * plane + o] = to_s<S, T>(g[i]);
                if (epi) {
                    const long long og = (long long)y * gd.pitch + x;
                    const T d = ux - snap[og];
                    snap[og] = ux;
                    acc.add(d * d, drho);
                }
            }
        }
        if (epi) {
            double a, bb;
            acc.block_total(a, bb, red);
            if (tid == 0) part = make_double2(a, bb);
        }
        // 3. the new set is complete (and every pull of the old one done):
        // this CTA's stores are visible to its own threads, then it arrives;
        // the next step waits for the others
        __syncthreads();
        cluster_arrive();
        b ^= 1;
        if (epi) {
            cluster_wait();  // every CTA's partial sums are written
            if (tid == 0) {
                double a = 0.0, m = 0.0;
                for (int r = 0; r < nc; r++) {  // rank order: the same sums in every CTA
                    const double2 p = *cl.map_shared_rank(&part, r);
                    a += p.x;
                    m += p.y;
                }
                const double res = sqrt(a), mass = nnodes + m;
                int stop = 0;
                if (!isfinite(res) || !isfinite(mass)) stop = 2;
                else if (res < st->tol) stop = 1;
                sh_stop = stop;
                if (rank == 0) {
                    st->res_step = t;
                    st->res = res;
                    st->mass = mass;
                    if (stop == 2) st->diverged = 1;
                    if (stop == 1) st->converged = 1;
                    if (stop) st->stop = 1;
                }
            }
            __syncthreads();  // sh_stop is visible to every thread
            if (sh_stop) {  // the same decision in every CTA
                done++;
                waited = true;
                break;
            }
            cluster_arrive();  // matched by the wait at the top of the next step
        }
    }
    if (!waited) cluster_wait();  // every CTA is done with this CTA's shared memory
    // write the slab of the final state
    const long long tend = t0 + done;
    S *pout = const_cast<S *>((tend & 1) ? pop1 : pop0);
    for (int i = 0; i < 9; i++)
        for (int q = tid; q < nslab; q += nthr) {
            const int ly = q / nx, x = q - ly * nx;
            pout[(long long)i * gd.plane + (long long)(v.y_lo + ly) * gd.pitch + x] =
                (b ? F1 : F0)[i * plane + ly * nx + x];
        }
}

}  // namespace prc
