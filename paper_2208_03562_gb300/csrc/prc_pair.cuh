// prc_pair.cuh -- the wall-aware general tile body with the collision in
// packed FP32x2 arithmetic (FP32 / FP16 storage): 64 x 8 nodes per 256-thread
// CTA, one pair of neighbouring nodes (x, x + 1), x even, per thread.  It is
// the general kernel of FP32 / FP16 handles and the tile body of the batch
// engine for those formats.
//
// Per node it does exactly what general_tile does (pull-streaming with
// bounce-back and the lid, density tile with a one-node ring per reading A1,
// density gradient, collision, store, residual terms); only the collision of
// the two nodes runs as one packed instruction stream.  Pairs whose nine
// sources lie inside the domain, away from the walls and the periodic seams,
// pull through three row pointers, with one aligned two-element load for the
// three planes of e_x = 0.
#pragma once

#include "prc_kernels.cuh"

namespace prc {

constexpr int PTW = 64, PTH = 8;               // pair tile: nodes
constexpr int PAIR_RW = PTW + 4;               // density-tile row: node lx at column lx + 2
constexpr int PAIR_SRHO = PAIR_RW * (PTH + 2);  // floats of the density tile (+ ring)

// Two neighbouring elements (first one at an even index) of global memory.
template <typename S>
struct PairG;
template <>
struct PairG<float> {
    template <bool CG>
    static __device__ __forceinline__ F2 ld(const float *p)
    {
        const float2 *q = reinterpret_cast<const float2 *>(p);
        return F2(CG ? __ldcg(q) : __ldg(q));
    }
    static __device__ __forceinline__ void st(float *p, F2 v) { *reinterpret_cast<float2 *>(p) = v.v; }
};
template <>
struct PairG<__half> {
    template <bool CG>
    static __device__ __forceinline__ F2 ld(const __half *p)
    {
        const __half2 *q = reinterpret_cast<const __half2 *>(p);
        return F2(__half22float2(CG ? __ldcg(q) : __ldg(q)));
    }
    static __device__ __forceinline__ void st(__half *p, F2 v)
    {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.v.x, v.v.y);
    }
};

// map_node for the tile's nodes and its ring (at most one node before the
// grid, any number after it in a partial tile): a conditional wrap instead of
// a remainder.  Coordinates within one grid length of the grid map exactly as
// in map_node; farther ones (nodes of a partial tile that no stored node
// uses) are clamped into the grid.
__device__ __forceinline__ void map_node_near(const Grid &gd, int &x, int &y)
{
    if (gd.bc >= 1) x = x < 0 ? x + gd.nx : (x >= gd.nx ? x - gd.nx : x);
    x = min(max(x, 0), gd.nx - 1);
    if (gd.bc == 2) y = y < 0 ? y + gd.ny : (y >= gd.ny ? y - gd.ny : y);
    y = min(max(y, 0), gd.ny - 1);
}

// The nine pulls of node (x, y) of the grid: fixed offsets from the node when
// every source lies inside the grid (no wall, no periodic seam), else pull9
// with the walls and the lid.  Either way the same values as pull9.
template <typename S, bool CG>
__device__ __forceinline__ void pull9_any(const S *__restrict__ src, const Grid &gd, int x, int y, float lid,
                                          float g[9])
{
    if ((x >= 1) & (x <= gd.nx - 2) & (y >= 1) & (y <= gd.ny - 2)) {
        const S *c = src + (long long)y * gd.pitch + x;
#pragma unroll
        for (int i = 0; i < 9; i++)
            g[i] = ld_pop<CG, S, float>(c + (long long)i * gd.plane - (long long)ey_of(i) * gd.pitch - ex_of(i));
    } else {
        pull9<S, float, CG>(src, gd, x, y, lid, g);
    }
}

// One fused time step on the 64 x 8 tile at (x0, y0) (x0 a multiple of 64);
// all 256 threads of the CTA call it.  srho holds PAIR_SRHO floats.
template <typename S, bool DRHO, bool EPI, bool FORCE, bool CG, bool RAW>
__device__ __forceinline__ void pair_tile(const S *__restrict__ src, S *__restrict__ dst, const Grid &gd,
                                          const Coef<float> &kf, const Coef<F2> &k2, float *__restrict__ snap,
                                          int x0, int y0, RedAcc<float> &acc, float *srho)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int px = tid & 31, ty = tid >> 5;
    const int xa = x0 + 2 * px, y = y0 + ty;  // the pair's first node
    const bool v0 = (xa < gd.nx) & (y < gd.ny), v1 = (xa + 1 < gd.nx) & (y < gd.ny);
    const long long o = (long long)y * gd.pitch + xa;
    float2 snap_old = make_float2(0.f, 0.f);
    if constexpr (EPI) {  // issue early: overlaps the pulls
        if (v1) snap_old = __ldcs(reinterpret_cast<const float2 *>(snap + o));
        else if (v0) snap_old.x = __ldcs(snap + o);
    }

    F2 g[9];
    const bool fast = (xa >= 1) & (xa + 2 <= gd.nx - 1) & (y >= 1) & (y <= gd.ny - 2);
    if (fast) {
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const S *row = src + (long long)i * gd.plane + (long long)(y - ey_of(i)) * gd.pitch + xa;
            if (ex_of(i) == 0) g[i] = PairG<S>::template ld<CG>(row);
            else g[i] = F2(ld_pop<CG, S, float>(row - ex_of(i)), ld_pop<CG, S, float>(row + 1 - ex_of(i)));
        }
    } else {
        // per node, at the node that stands in for it outside the grid
        float ga[9], gb[9];
        int mx = xa, my = y;
        map_node_near(gd, mx, my);
        pull9_any<S, CG>(src, gd, mx, my, kf.lid, ga);
        mx = xa + 1;
        my = y;
        map_node_near(gd, mx, my);
        pull9_any<S, CG>(src, gd, mx, my, kf.lid, gb);
#pragma unroll
        for (int i = 0; i < 9; i++) g[i] = F2(ga[i], gb[i]);
    }

    F2 dxr(0.f), dyr(0.f);
    if constexpr (DRHO) {
        constexpr int RW = PAIR_RW;
        *reinterpret_cast<float2 *>(srho + (ty + 1) * RW + 2 * px + 2) = sum9(g).v;
        constexpr int nring = 2 * (PTW + 2) + 2 * PTH;
        if (tid < nring) {
            int lx, ly;
            if (tid < PTW + 2) { lx = tid - 1; ly = -1; }
            else if (tid < 2 * (PTW + 2)) { lx = tid - (PTW + 2) - 1; ly = PTH; }
            else if (tid < 2 * (PTW + 2) + PTH) { lx = -1; ly = tid - 2 * (PTW + 2); }
            else { lx = PTW; ly = tid - 2 * (PTW + 2) - PTH; }
            int gx = x0 + lx, gy = y0 + ly;
            map_node_near(gd, gx, gy);
            float gr[9];
            pull9_any<S, CG>(src, gd, gx, gy, kf.lid, gr);
            srho[(ly + 1) * RW + lx + 2] = sum9(gr);
        }
        __syncthreads();
        float dx[2], dy[2];
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const float *c = srho + (ty + 1) * RW + 2 * px + 2 + j;
            const float rE = c[1], rW = c[-1];
            const float rN = c[RW], rS = c[-RW];
            const float rNE = c[RW + 1], rNW = c[RW - 1];
            const float rSE = c[-RW + 1], rSW = c[-RW - 1];
            drho_stencil<float>(rE, rW, rN, rS, rNE, rNW, rSE, rSW, kf.inv12, kf.inv12r, dx[j], dy[j]);
        }
        dxr = F2(dx[0], dx[1]);
        dyr = F2(dy[0], dy[1]);
        __syncthreads();  // srho may be refilled by the next tile of this CTA
    }

    F2 ux, uy, drho;
    collide<F2, DRHO, FORCE, RAW>(k2, g, dxr, dyr, ux, uy, drho);
    if (v1) {
#pragma unroll
        for (int i = 0; i < 9; i++) PairG<S>::st(dst + (long long)i * gd.plane + o, g[i]);
    } else if (v0) {
#pragma unroll
        for (int i = 0; i < 9; i++) dst[(long long)i * gd.plane + o] = to_s<S, float>(g[i].v.x);
    }
    if constexpr (EPI) {
        if (v0) {
            const float d = ux.v.x - snap_old.x;
            acc.add(d * d, drho.v.x);
        }
        if (v1) {
            const float d = ux.v.y - snap_old.y;
            acc.add(d * d, drho.v.y);
            __stcs(reinterpret_cast<float2 *>(snap + o), ux.v);
        } else if (v0) {
            __stcs(snap + o, ux.v.x);
        }
    }
}

// One fused time step of the whole grid (general kernel for FP32 / FP16):
// one 64 x 8 tile per CTA over the single rectangle of `rc`; the CTA totals
// of a residual step go to partials[part0 + blockIdx.x].
template <typename S, bool DRHO, bool EPI, bool FORCE, bool RAW>
__global__ void __launch_bounds__(256, 4)
k_step_pair(const S *__restrict__ src, S *__restrict__ dst, Grid gd, Coef<float> kf, Coef<F2> k2,
            float *__restrict__ snap, double2 *__restrict__ partials, const DevStatus *__restrict__ st,
            const __grid_constant__ Rects rc, int part0)
{
    if (st->stop) return;
    __shared__ __align__(16) float srho[PAIR_SRHO];
    const int e = blockIdx.x;
    const int x0 = rc.x0[0] + (e % rc.tiles_x[0]) * PTW, y0 = rc.y0[0] + (e / rc.tiles_x[0]) * PTH;
    RedAcc<float> acc;
    pair_tile<S, DRHO, EPI, FORCE, false, RAW>(src, dst, gd, kf, k2, snap, x0, y0, acc, srho);
    if constexpr (EPI) {
        __shared__ double red[2 * (256 / 32)];
        double a, b;
        acc.block_total(a, b, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[part0 + blockIdx.x] = make_double2(a, b);
    }
}

}  // namespace prc
