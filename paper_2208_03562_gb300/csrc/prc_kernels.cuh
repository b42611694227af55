// prc_kernels.cuh -- kernels of the single-instance path, templated on the
// storage type S (double, float, __half) and the collision type T.
#pragma once

#include "prc_device.cuh"
#include "prc_reduce.cuh"

namespace prc {

constexpr int BX = 32;  // default tile width  (nodes, one per thread)
constexpr int BY = 8;   // default tile height
constexpr int MAX_RECTS = 4;

// Rectangles of nodes handled by the general tile body (the whole domain, or
// the edge strips around the interior tiles of the TMA kernel), enumerated as
// a 1-D list of tiles.  Each rectangle has its own tile shape: 2^lw nodes wide
// and (CTA threads) >> lw high, so that thin strips are covered without idle
// threads.
struct Rects {
    int n;
    int x0[MAX_RECTS], y0[MAX_RECTS], x1[MAX_RECTS], y1[MAX_RECTS];
    int lw[MAX_RECTS];       // log2 of the tile width
    int tiles_x[MAX_RECTS];
    int start[MAX_RECTS + 1];  // first tile index of each rectangle; start[n] = total
};

// Floats of density tile (+ ring) that general_tile needs for a CTA of
// `threads` threads and any tile width 2 <= 2^lw <= threads / 2.
__host__ __device__ constexpr int srho_floats(int threads) { return 4 * (threads / 2 + 2); }

// Origin and shape of tile `e` of the rectangle list.
__device__ __forceinline__ void rect_tile(const Rects &rc, int e, int &x0, int &y0, int &x1, int &y1, int &lw)
{
    int r = 0;
    while (r + 1 < rc.n && e >= rc.start[r + 1]) r++;
    const int lt = e - rc.start[r];
    lw = rc.lw[r];
    const int th = (int)(blockDim.x * blockDim.y) >> lw;
    x0 = rc.x0[r] + (lt % rc.tiles_x[r]) * (1 << lw);
    y0 = rc.y0[r] + (lt / rc.tiles_x[r]) * th;
    x1 = rc.x1[r];
    y1 = rc.y1[r];
}

// One fused time step on one tile of 2^lw x (threads >> lw) nodes at (x0, y0)
// of the nodes x < x1, y < y1 (all threads of the CTA call it): pull-stream +
// walls, density tile (+1 ring) in shared memory `srho` (srho_floats(threads)
// values of type T) for the density gradient, collision, store.  With EPI the
// thread adds (u_x - u_x,snapshot)^2 and drho of its node to `acc` and
// refreshes the snapshot (residual of Sec. 5.2).
template <typename S, typename T, bool DRHO, bool EPI, bool FORCE, bool CG = false, bool RAW = false>
__device__ __forceinline__ void general_tile(const S *__restrict__ src, S *__restrict__ dst, const Grid &gd,
                                             const Coef<T> &k, T *__restrict__ snap, int x0, int y0, int x1, int y1,
                                             int lw, RedAcc<T> &acc, T *srho)
{
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int tw = 1 << lw, th = nthr >> lw;
    const int tx = tid & (tw - 1), ty = tid >> lw;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = (x < x1) & (y < y1);
    T snap_old = T(0);
    if constexpr (EPI) {  // issue early: overlaps the pulls
        if (valid) snap_old = __ldcs(snap + (long long)y * gd.pitch + x);
    }

    T g[9];
    int mx = x, my = y;
    map_node(gd, mx, my);
    pull9<S, T, CG>(src, gd, mx, my, k.lid, g);

    T dxr = T(0), dyr = T(0);
    if constexpr (DRHO) {
        const int RW = tw + 2;
        srho[(ty + 1) * RW + tx + 1] = sum9(g);
        const int nring = 2 * RW + 2 * th;
        for (int q = tid; q < nring; q += nthr) {
            int lx, ly;
            if (q < RW) { lx = q; ly = 0; }
            else if (q < 2 * RW) { lx = q - RW; ly = th + 1; }
            else if (q < 2 * RW + th) { lx = 0; ly = q - 2 * RW + 1; }
            else { lx = tw + 1; ly = q - 2 * RW - th + 1; }
            int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            map_node(gd, gx, gy);
            T gr[9];
            pull9<S, T, CG>(src, gd, gx, gy, k.lid, gr);
            srho[ly * RW + lx] = sum9(gr);
        }
        __syncthreads();
        const T *c = srho + (ty + 1) * RW + tx + 1;
        const T rE = c[1], rW = c[-1];
        const T rN = c[RW], rS = c[-RW];
        const T rNE = c[RW + 1], rNW = c[RW - 1];
        const T rSE = c[-RW + 1], rSW = c[-RW - 1];
        drho_stencil<T>(rE, rW, rN, rS, rNE, rNW, rSE, rSW, k.inv12, k.inv12r, dxr, dyr);
        __syncthreads();  // srho may be refilled by the next tile of this CTA
    }

    T ux = T(0), uy = T(0), drho = T(0);
    if (valid) {
        collide<T, DRHO, FORCE, RAW>(k, g, dxr, dyr, ux, uy, drho);
        const long long o = (long long)y * gd.pitch + x;
#pragma unroll
        for (int i = 0; i < 9; i++) dst[(long long)i * gd.plane + o] = to_s<S, T>(g[i]);
        if constexpr (EPI) {
            const T d = ux - snap_old;
            __stcs(snap + o, ux);
            acc.add(d * d, drho);
        }
    }
}

// One fused time step on the nodes of `rc` (general kernel, one tile per
// CTA); the CTA totals of a residual step go to partials[part0 + blockIdx.x].
template <typename S, typename T, bool DRHO, bool EPI, bool FORCE, bool RAW>
__global__ void __launch_bounds__(BX * BY)
k_step(const S *__restrict__ src, S *__restrict__ dst, Grid gd, Coef<T> k, T *__restrict__ snap,
       double2 *__restrict__ partials, const DevStatus *__restrict__ st, const __grid_constant__ Rects rc, int part0)
{
    if (st->stop) return;
    __shared__ T srho[srho_floats(BX * BY)];
    int x0, y0, x1, y1, lw;
    rect_tile(rc, blockIdx.x, x0, y0, x1, y1, lw);
    RedAcc<T> acc;
    general_tile<S, T, DRHO, EPI, FORCE, false, RAW>(src, dst, gd, k, snap, x0, y0, x1, y1, lw, acc, srho);
    if constexpr (EPI) {
        __shared__ double red[2 * (BX * BY / 32)];
        double a, b;
        acc.block_total(a, b, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[part0 + blockIdx.x] = make_double2(a, b);
    }
}

// f~ = f^eq(rho, u) (Eq. 12, uncorrected), stored shifted; snapshot = u_x.
template <typename S, typename T>
__global__ void k_init_fields(S *__restrict__ dst, Grid gd, Coef<double> k, double gamma,
                              const double *__restrict__ rho_in, const double *__restrict__ ux_in,
                              const double *__restrict__ uy_in, T *__restrict__ snap)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= gd.nx || y >= gd.ny) return;
    const long long n = (long long)y * gd.nx + x;
    const double rho = rho_in[n], ux = ux_in[n], uy = uy_in[n];
    const double drho = rho - 1.0, ig = 1.0 / gamma;
    // raw equilibrium moments (rectangular) minus the rest-state moments
    const double D00 = drho, D10 = rho * ux, D01 = rho * uy;
    const double D20 = k.c2 * drho + rho * ux * ux * ig;
    const double D02 = k.c2 * drho + rho * uy * uy * ig;
    const double D11 = rho * ux * uy * ig;
    const double D21 = rho * (k.c2 + ux * ux * ig * ig) * uy;
    const double D12 = rho * (k.c2 + uy * uy * ig * ig) * ux;
    const double D22 = k.c4 * drho + rho * k.c2 * (ux * ux + uy * uy) + rho * ux * ux * uy * uy;
    const double ir = 1.0 / k.r;
    const double e01 = D01 * ir, e02 = D02 * k.inv_r2, e11 = D11 * ir;
    const double e21 = D21 * ir, e12 = D12 * k.inv_r2, e22 = D22 * k.inv_r2;
    double g[9];
    g[0] = D00 - D20 - e02 + e22;
    g[1] = 0.5 * (D10 + D20 - e12 - e22);
    g[2] = 0.5 * (e01 + e02 - e21 - e22);
    g[3] = 0.5 * (-D10 + D20 + e12 - e22);
    g[4] = 0.5 * (-e01 + e02 + e21 - e22);
    g[5] = 0.25 * (e11 + e21 + e12 + e22);
    g[6] = 0.25 * (-e11 + e21 - e12 + e22);
    g[7] = 0.25 * (e11 - e21 - e12 + e22);
    g[8] = 0.25 * (-e11 - e21 + e12 + e22);
    const long long o = (long long)y * gd.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; i++) dst[(long long)i * gd.plane + o] = to_s<S, T>((T)g[i]);
    snap[o] = (T)ux;
}

// Fields of the stored post-collision state: rho = 1 + sum g, rho u = sum g e
// - F / (2 gamma) (the rest state carries no momentum).
template <typename S, typename T>
__global__ void k_fields(const S *__restrict__ src, Grid gd, Coef<double> k, double *__restrict__ rho_out,
                         double *__restrict__ ux_out, double *__restrict__ uy_out, T *__restrict__ snap)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= gd.nx || y >= gd.ny) return;
    const long long o = (long long)y * gd.pitch + x;
    double g[9];
#pragma unroll
    for (int i = 0; i < 9; i++) g[i] = (double)ld_s<S, T>(src + (long long)i * gd.plane + o);
    const double s00 = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const double s10 = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const double s01 = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    const double rho = 1.0 + s00;
    const double ux = (s10 - k.hx) / rho, uy = (k.r * s01 - k.hy) / rho;
    const long long n = (long long)y * gd.nx + x;
    if (rho_out) rho_out[n] = rho;
    if (ux_out) ux_out[n] = ux;
    if (uy_out) uy_out[n] = uy;
    if (snap) snap[o] = (T)ux;
}

// Full FP64 populations <-> shifted storage.
template <typename S, typename T>
__global__ void k_set_pop(S *__restrict__ dst, Grid gd, Coef<double> k, const double *__restrict__ f)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= gd.nx || y >= gd.ny) return;
    const long long nn = (long long)gd.nx * gd.ny, n = (long long)y * gd.nx + x;
    const long long o = (long long)y * gd.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; i++) dst[(long long)i * gd.plane + o] = to_s<S, T>((T)(f[i * nn + n] - k.w[i]));
}

template <typename S, typename T>
__global__ void k_get_pop(const S *__restrict__ src, Grid gd, Coef<double> k, double *__restrict__ f)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= gd.nx || y >= gd.ny) return;
    const long long nn = (long long)gd.nx * gd.ny, n = (long long)y * gd.nx + x;
    const long long o = (long long)y * gd.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; i++) f[i * nn + n] = (double)ld_s<S, T>(src + (long long)i * gd.plane + o) + k.w[i];
}

// Uniform density shift: f_i += w_i(r) delta at every node (the rest
// populations carry density and no momentum), rounded to the storage.
template <typename S, typename T>
__global__ void k_add_rest(S *__restrict__ pop, Grid gd, Coef<double> k, double delta)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= gd.nx || y >= gd.ny) return;
    const long long o = (long long)y * gd.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        S *p = pop + (long long)i * gd.plane + o;
        *p = to_s<S, T>((T)((double)ld_s<S, T>(p) + k.w[i] * delta));
    }
}

// Per-CTA FP64 partial sums of sum_i g_i (total mass minus the node count).
template <typename S, typename T>
__global__ void __launch_bounds__(BX * BY) k_mass_partial(const S *__restrict__ src, Grid gd, double2 *__restrict__ partials)
{
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    double dm = 0.0, z = 0.0;
    if (x < gd.nx && y < gd.ny) {
        const long long o = (long long)y * gd.pitch + x;
#pragma unroll
        for (int i = 0; i < 9; i++) dm += (double)ld_s<S, T>(src + (long long)i * gd.plane + o);
    }
    __shared__ double red[2 * (BX * BY / 32)];
    RedAcc<double> acc;
    acc.add(z, dm);
    double a, b;
    acc.block_total(a, b, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = make_double2(a, b);
}

}  // namespace prc
