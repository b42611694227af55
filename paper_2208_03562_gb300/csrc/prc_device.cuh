// prc_device.cuh -- device-side building blocks of the fused PRC-LBM step.
//
// Storage: nine SoA planes g_i[y][x] = f~_i - w_i(r) rho0 (post-collision
// populations shifted by the rest state, rho0 = 1), row pitch `pitch`
// elements, plane stride `plane` elements.  Shifting keeps FP32/FP16 storage
// precision on the small deviations, and the collision below is written in
// deviation form so that no O(1) quantity is ever subtracted from another.
//
// The collision is the App. A sequence of arXiv:2208.03562 (raw moments,
// scaling S, central moments F, relaxation to the gamma-preconditioned
// equilibria of Eq. 14 with the corrections of Eqs. 38-40 and the local strain
// rates of Eqs. 43-48, F^-1, S^-1, P^-1) with the algebra rearranged:
//   * only the central moments that are relaxed with a rate other than 1 are
//     formed (k20, k02, k11); k21, k12, k22 and k10, k01 are replaced by
//     their post-collision values directly (omega_21 = omega_12 = omega_22 =
//     omega_1 = 1, App. A; k~10 = F_x / (2 gamma) for any omega_1);
//   * the non-equilibrium parts n_2s, n_2d, n_11 are formed from the
//     deviation moments of g, e.g. n_20 = s20 - c^2 drho - rho u_x^2 / gamma
//     + 2 u_x h_x;
//   * post-collision raw moments are assembled minus the rest-state moments
//     (1, 0, 0, c^2, c^2, 0, 0, 0, c^4), so P^-1 S^-1 of them is g~ directly.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace prc {

// Per-instance constants, precomputed on the host in FP64 and cast to the
// collision precision T.
template <typename T>
struct Coef {
    T r, r2, inv_r, inv_r2;   // aspect ratio r = dy/dx and powers
    T c2, c4;                 // c^2 = q^2 c_s*^2, q = min(1, r) (Eq. 2)
    T w_nu, w_xi;             // shear / bulk relaxation rates
    T one_m_w_nu, one_m_w_xi; // 1 - omega
    T src_nu, src_xi;         // 1 - omega / 2
    T m2tau_nu, m2tau_xi;     // -2 (1/omega - 1/2)
    T mtau_nu;                // -(1/omega_nu - 1/2)
    T ig, h1, a3, Pg, Qg;     // 1/g, 1/g - 1, 1/g^2 - 3/g + 2, P_gamma, Q_gamma
    T hPg, hQg;               // P_gamma / 2, Q_gamma / 2
    T Ax, By;                 // A = Ax u_x, B = By u_y (Eq. 43)
    T k3x, k3y;               // (3c^2 - 1)/2, (3c^2 - r^2)/2
    T Cb0, Cs0;               // -2 c^2 / omega_xi, -2 c^2 / omega_nu
    T h1c2;                   // (1/g - 1) c^2
    T hx, hy;                 // F / (2 gamma): half-force velocity shift
    T twoQFx, twoQFy;         // 2 Q_gamma F (source moments, Eq. 13-central)
    T QFx, QFy;               // Q_gamma F
    T lid;                    // c^2 U / (2 r^2): moving-lid bounce-back term
    T inv12, inv12r;          // 1/12, 1/(12 r): density-gradient stencil
    T w[9];                   // rest populations w_i(r)
};

struct Grid {
    int nx, ny;
    int pitch;        // elements per row
    int bc;           // 0 cavity, 1 channel (x-periodic), 2 periodic
    long long plane;  // elements per plane
    int lid_on;       // top wall moves
    int pad;
};

// Device-side run status (one per instance).
struct DevStatus {
    int stop;          // 1: later step kernels exit at entry
    int converged;
    int diverged;
    int timeout;
    long long res_step;  // step of the last residual evaluation
    double tol;          // lbm_run target (<= 0: never stop)
    double res;          // last residual (FP64)
    double mass;         // total mass at the last evaluation
    double mass_now;     // result of the on-demand mass reduction
};

// velocity set (Eq. 3): e_x and e_y / r, opposite directions
__host__ __device__ constexpr int ex_of(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey_of(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5); }

// storage <-> collision precision
template <typename S, typename T> __device__ __forceinline__ T ld_s(const S *p);
template <> __device__ __forceinline__ double ld_s<double, double>(const double *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_s<float, float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_s<__half, float>(const __half *p) { return __half2float(__ldg(p)); }

template <typename S, typename T> __device__ __forceinline__ S to_s(T v);
template <> __device__ __forceinline__ double to_s<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_s<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_s<__half, float>(float v) { return __float2half_rn(v); }

template <typename T> __device__ __forceinline__ T rcp(T v);
template <> __device__ __forceinline__ double rcp<double>(double v) { return 1.0 / v; }
template <> __device__ __forceinline__ float rcp<float>(float v) { return __frcp_rn(v); }

// Map a node coordinate to the node whose density stands in for it (reading
// A1: nearest fluid node across a wall, wrap across a periodic direction).
__device__ __forceinline__ void map_node(const Grid &gd, int &x, int &y)
{
    if (gd.bc >= 1) x = (x + gd.nx) % gd.nx;
    else x = min(max(x, 0), gd.nx - 1);
    if (gd.bc == 2) y = (y + gd.ny) % gd.ny;
    else y = min(max(y, 0), gd.ny - 1);
}

// Pull-streaming f_i(x, t+1) = f~_i(x - e_i, t) (App. A) with half-way
// bounce-back: a source outside a wall is replaced by the opposite population
// of the node itself, plus the moving-top-wall term -/+ c^2 U / (2 r^2) on the
// two diagonal links that come from above (directions SW, SE).
template <typename S, typename T>
__device__ __forceinline__ void pull9(const S *__restrict__ src, const Grid &gd, int x, int y, T lid, T g[9])
{
#pragma unroll
    for (int i = 0; i < 9; i++) {
        int sx = x - ex_of(i), sy = y - ey_of(i);
        if (gd.bc >= 1) sx = sx < 0 ? sx + gd.nx : (sx >= gd.nx ? sx - gd.nx : sx);
        if (gd.bc == 2) sy = sy < 0 ? sy + gd.ny : (sy >= gd.ny ? sy - gd.ny : sy);
        bool inside = (sx >= 0) & (sx < gd.nx) & (sy >= 0) & (sy < gd.ny);
        if (inside) {
            g[i] = ld_s<S, T>(src + (long long)i * gd.plane + (long long)sy * gd.pitch + sx);
        } else {
            T v = ld_s<S, T>(src + (long long)opp_of(i) * gd.plane + (long long)y * gd.pitch + x);
            if (sy >= gd.ny && gd.lid_on) {
                if (i == 7) v -= lid;
                if (i == 8) v += lid;
            }
            g[i] = v;
        }
    }
}

template <typename T>
__device__ __forceinline__ T sum9(const T g[9])
{
    return ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
}

// The collision in deviation form.  In: g[9] streamed shifted populations,
// density gradient (dxr, dyr).  Out: g[9] post-collision shifted populations;
// u_x, u_y, drho of the node.
template <typename T, bool DRHO>
__device__ __forceinline__ void collide(const Coef<T> &k, T g[9], T dxr, T dyr, T &ux_out, T &uy_out, T &drho_out)
{
    // square-lattice raw moments of the deviations (Eq. 62 applied to g)
    const T s00 = sum9(g);
    const T s10 = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const T s01 = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    const T d58 = (g[5] + g[6]) + (g[7] + g[8]);
    const T s20 = (g[1] + g[3]) + d58;
    const T s02 = (g[2] + g[4]) + d58;
    const T s11 = (g[5] - g[6]) + (g[7] - g[8]);

    // hydrodynamic fields (rho u = sum f e + F / (2 gamma))
    const T rho = T(1) + s00;
    const T irho = rcp<T>(rho);
    const T jx = s10 + k.hx;
    const T jy = k.r * s01 + k.hy;
    const T ux = jx * irho, uy = jy * irho;
    const T ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const T rux2 = rho * ux2, ruy2 = rho * uy2, ruxy = rho * uxy;

    // non-equilibrium central moments w.r.t. the base equilibria of Eq. 14
    const T n20 = s20 - k.c2 * s00 - k.ig * rux2 + T(2) * ux * k.hx;
    const T n02 = k.r2 * s02 - k.c2 * s00 - k.ig * ruy2 + T(2) * uy * k.hy;
    const T n11 = k.r * s11 - k.ig * ruxy + uy * k.hx + ux * k.hy;
    const T n2s = n20 + n02, n2d = n20 - n02;

    // local strain rates (Eqs. 43-48, R per Eq. 45)
    T ebr = T(0), esr = T(0);
    if (DRHO) {
        const T A = k.Ax * ux, B = k.By * uy;
        ebr = -A * dxr - B * dyr;
        esr = -A * dxr + B * dyr;
    }
    const T R2s = n2s + ebr, R2d = n2d + esr;
    const T Px = k.hPg * ux2, Py = k.hPg * uy2, Qx = k.hQg * ux2, Qy = k.hQg * uy2;
    const T ax = (Px + Qy + k.k3x) * rho;
    const T ay = (Py + Qx + k.k3y) * rho;
    const T dx = (Px - Qy + k.k3x) * rho;
    const T dy = (Py - Qx + k.k3y) * rho;
    const T Cbx = k.Cb0 * rho + ax, Cby = k.Cb0 * rho + ay;
    const T Csx = k.Cs0 * rho + dx, Csy = -k.Cs0 * rho - dy;
    const T X = (Csy * R2s - Cby * R2d) * rcp<T>(Cbx * Csy - Csx * Cby);
    const T Y = (R2s - Cbx * X) * rcp<T>(Cby);

    // corrections of the extended equilibria (Eqs. 30, 38-40 / App. A)
    const T corr_s = k.m2tau_xi * (ax * X + ay * Y - ebr);
    const T corr_d = k.m2tau_nu * (dx * X - dy * Y - esr);
    T c11 = k.Qg * ruxy * (X + Y);
    if (DRHO) c11 += k.h1c2 * (uy * dxr + ux * dyr);
    const T corr_11 = k.mtau_nu * c11;

    // central source moments (Eq. 13-central)
    const T sig2s = k.twoQFx * ux + k.twoQFy * uy;
    const T sig2d = k.twoQFx * ux - k.twoQFy * uy;
    const T sig11 = k.QFx * uy + k.QFy * ux;

    // relaxation (App. A); dt2s = k~2s - 2 c^2 rho
    const T dt2s = k.h1 * (rux2 + ruy2) + k.one_m_w_xi * n2s + k.w_xi * corr_s + k.src_xi * sig2s;
    const T t2d = k.h1 * (rux2 - ruy2) + k.one_m_w_nu * n2d + k.w_nu * corr_d + k.src_nu * sig2d;
    const T t11 = k.h1 * ruxy + k.one_m_w_nu * n11 + k.w_nu * corr_11 + k.src_nu * sig11;
    const T dt20 = T(0.5) * (dt2s + t2d);  // k~20 - c^2 rho
    const T dt02 = T(0.5) * (dt2s - t2d);  // k~02 - c^2 rho
    const T t21 = k.a3 * rux2 * uy;
    const T t12 = k.a3 * ruy2 * ux;
    const T t20 = k.c2 * rho + dt20, t02 = k.c2 * rho + dt02;

    // post-collision raw moments minus the rest-state moments (F^-1)
    const T D00 = s00;
    const T D10 = jx + k.hx;
    const T D01 = jy + k.hy;
    const T D20 = k.c2 * s00 + dt20 + T(2) * ux * k.hx + rux2;
    const T D02 = k.c2 * s00 + dt02 + T(2) * uy * k.hy + ruy2;
    const T D11 = t11 + uy * k.hx + ux * k.hy + ruxy;
    const T D21 = t21 + T(2) * ux * t11 + ux2 * k.hy + uy * t20 + T(2) * uxy * k.hx + rux2 * uy;
    const T D12 = t12 + T(2) * uy * t11 + uy2 * k.hx + ux * t02 + T(2) * uxy * k.hy + ruy2 * ux;
    const T D22 = k.c4 * s00 + T(2) * ux * t12 + ux2 * t02 + T(2) * uy * t21 + T(4) * uxy * t11
                + T(2) * ux2 * uy * k.hy + uy2 * t20 + T(2) * ux * uy2 * k.hx + rux2 * uy2;

    // S^-1 then P^-1 (Eq. 72)
    const T e01 = D01 * k.inv_r, e02 = D02 * k.inv_r2, e11 = D11 * k.inv_r;
    const T e21 = D21 * k.inv_r, e12 = D12 * k.inv_r2, e22 = D22 * k.inv_r2;
    g[0] = (D00 - D20) + (e22 - e02);
    const T a1 = T(0.5) * (D20 - e22), b1 = T(0.5) * (D10 - e12);
    g[1] = a1 + b1;
    g[3] = a1 - b1;
    const T a2 = T(0.5) * (e02 - e22), b2 = T(0.5) * (e01 - e21);
    g[2] = a2 + b2;
    g[4] = a2 - b2;
    const T p = T(0.25) * (e21 + e22), m = T(0.25) * (e11 + e12);
    const T pp = T(0.25) * (e22 - e21), mm = T(0.25) * (e11 - e12);
    g[5] = p + m;
    g[6] = p - m;
    g[7] = pp + mm;
    g[8] = pp - mm;

    ux_out = ux;
    uy_out = uy;
    drho_out = s00;
}

}  // namespace prc
