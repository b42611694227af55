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
//   * the strain-rate system of Eqs. 43-44 is solved for rho (X + Y) and
//     rho (X - Y), the only combinations the relaxed moments use (see the
//     comments in collide);
//   * post-collision raw moments are assembled minus the rest-state moments
//     (1, 0, 0, c^2, c^2, 0, 0, 0, c^4), so P^-1 S^-1 of them is g~ directly.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "prc_vec.cuh"

namespace prc {

// Per-instance constants, precomputed on the host in FP64 and cast to the
// collision type T (float, double, or F2 with both lanes equal).
template <typename T>
struct Coef {
    T r, r2;                   // aspect ratio r = dy/dx, r^2
    T c2, c4;                  // c^2 = q^2 c_s*^2, q = min(1, r) (Eq. 2); c^4
    T hh1;                     // (1/g - 1)/2
    T Ax, By;                  // A = Ax u_x, B = By u_y (Eq. 43)
    T pp, npp, pm;             // (P_gamma + Q_gamma)/4, its negation, (P_gamma - Q_gamma)/4
    T e1, e2, ne2, e3;         // strain-rate system constants: Cb0 + k3, k3d, -k3d, Cs0 + k3
    T kS, kD;                  // omega_xi tau_xi Cb0, omega_nu tau_nu Cs0
    T h1x2, omw2;              // 2 (1/g - 1), 2 (1 - omega_nu)
    T kdQg2, kdh1c2x2;         // -2 omega_nu tau_nu Q_gamma, -2 omega_nu tau_nu (1/g - 1) c^2
    T a3p1, a34p1;             // a3 + 1, 4 a3 + 1 with a3 = 1/g^2 - 3/g + 2
    T qr, qr2, hr, hr2, inv_r2;  // 1/(4r), 1/(4r^2), 1/(2r), 1/(2r^2), 1/r^2
    T n2qr, n2qr2;             // -1/(2r), -1/(2r^2)
    T hx, hy;                  // F / (2 gamma): half-force velocity shift
    T fsx, fsy, fdx, nfdy;     // (1 - omega/2) Q_gamma F: source moments (Eq. 13-central)
    T fdx2, fdy2;              // 2 fdx, 2 fdy
    T nig, nr2, ninv_r2;       // -1/g, -r^2, -1/r^2
    T lid;                     // c^2 U / (2 r^2): moving-lid bounce-back term
    T ig2;                     // 1 / g^2 (raw-moment scheme)
    T inv12, inv12r;           // 1/12, 1/(12 r): density-gradient stencil
    T w[9];                    // rest populations w_i(r)
};

struct Grid {
    int nx, ny;
    int pitch;        // elements per row
    int bc;           // 0 cavity, 1 channel (x-periodic), 2 periodic
    long long plane;  // elements per plane
    int lid_on;       // top wall moves
    int model;        // 0: central moments (PRC-LBM); 1: raw moments (PRNR-LBM)
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

// L2-coherent loads (ld.global.cg) for data written by other CTAs of the same
// persistent launch
template <typename S, typename T> __device__ __forceinline__ T ld_cg(const S *p);
template <> __device__ __forceinline__ double ld_cg<double, double>(const double *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ld_cg<float, float>(const float *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ld_cg<__half, float>(const __half *p) { return __half2float(__ldcg(p)); }

template <bool CG, typename S, typename T>
__device__ __forceinline__ T ld_pop(const S *p)
{
    if constexpr (CG) return ld_cg<S, T>(p);
    else return ld_s<S, T>(p);
}

template <typename S, typename T> __device__ __forceinline__ S to_s(T v);
template <> __device__ __forceinline__ double to_s<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_s<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_s<__half, float>(float v) { return __float2half_rn(v); }


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
template <typename S, typename T, bool CG = false>
__device__ __forceinline__ void pull9(const S *__restrict__ src, const Grid &gd, int x, int y, T lid, T g[9])
{
#pragma unroll
    for (int i = 0; i < 9; i++) {
        int sx = x - ex_of(i), sy = y - ey_of(i);
        if (gd.bc >= 1) sx = sx < 0 ? sx + gd.nx : (sx >= gd.nx ? sx - gd.nx : sx);
        if (gd.bc == 2) sy = sy < 0 ? sy + gd.ny : (sy >= gd.ny ? sy - gd.ny : sy);
        bool inside = (sx >= 0) & (sx < gd.nx) & (sy >= 0) & (sy < gd.ny);
        if (inside) {
            g[i] = ld_pop<CG, S, T>(src + (long long)i * gd.plane + (long long)sy * gd.pitch + sx);
        } else {
            T v = ld_pop<CG, S, T>(src + (long long)opp_of(i) * gd.plane + (long long)y * gd.pitch + x);
            if (sy >= gd.ny && gd.lid_on) {
                if (i == 7) v -= lid;
                if (i == 8) v += lid;
            }
            g[i] = v;
        }
    }
}

// Density deviation sum_i g_i, summed in the order the collision forms s00
// (same operands, same pairing), so that a kernel which takes the density
// before a barrier and collides after it computes those sums once.
template <typename T>
PRC_HD T sum9(const T g[9])
{
    const T p13 = vadd(g[1], g[3]), p24 = vadd(g[2], g[4]);
    const T d58 = vadd(vadd(g[5], g[6]), vadd(g[7], g[8]));
    return vadd(vadd(g[0], d58), vadd(p13, p24));
}

// Density gradients of reading A1 from the eight neighbour densities,
// dx = [4 (rE - rW) + (rNE - rNW) + (rSE - rSW)] / 12 and
// dy = [4 (rN - rS) + (rNE - rSE) + (rNW - rSW)] / (12 r), in a fixed sequence
// of explicitly rounded operations, so that every kernel (scalar or packed
// lanes) forms the same value for a node.
template <typename T>
PRC_HD void drho_stencil(T rE, T rW, T rN, T rS, T rNE, T rNW, T rSE, T rSW, T i12, T i12r, T &dx, T &dy)
{
    dx = vmul(vadd(vfma(splat<T>(4.0), vsub(rE, rW), vsub(rNE, rNW)), vsub(rSE, rSW)), i12);
    dy = vmul(vadd(vfma(splat<T>(4.0), vsub(rN, rS), vsub(rNE, rSE)), vsub(rNW, rSW)), i12r);
}

// The collision in deviation form (App. A with the algebra rearranged as in
// the file header), generic over float, double and packed F2.
// In: g[9] streamed shifted populations, density gradient (dxr, dyr).
// Out: g[9] post-collision shifted populations; u_x, u_y, drho of the node.
// RAW selects the raw-moment scheme (PRNR-LBM, Eq.
// LBErawmomentrectangularlattice, Sec. 5.3) instead of the central one: its
// post-collision raw moments of orders 0-2 are the same (the non-equilibrium
// second-order moments and the sources agree between the frames), and those
// of orders 3-4 are the raw equilibria of Eq. 12 (rates 1) instead of the
// binomial transform of the central ones.
//
// The collision falls into two halves: collide_moments forms everything that
// does not depend on the density gradient (moments, velocity, the
// non-equilibrium moments and the strain-rate system's matrix), and
// collide_relax the rest.  A kernel may run the first half while it waits for
// the densities of its neighbours; collide() is the two in sequence, the same
// operations in the same order.
template <typename T>
struct Moments {
    T s00, jx, jy, ux, uy;            // density deviation, momentum, velocity
    T ux2, uy2, uxy, rux2, ruy2, ruxy;  // their products
    T sp, sm, c2s00;                  // rho (u_x^2 +- u_y^2), c^2 s00
    T n2s, n2d, n11;                  // non-equilibrium second-order central moments
    T m11, m22, m12, nm21, idet;      // strain-rate system (see collide_moments)
};

template <typename T, bool FORCE>
PRC_HD void collide_moments(const Coef<T> &k, const T g[9], Moments<T> &M)
{
    // square-lattice raw moments of the deviations (Eq. 62 applied to g)
    const T a13 = vsub(g[1], g[3]), a56 = vsub(g[5], g[6]), a87 = vsub(g[8], g[7]);
    const T p13 = vadd(g[1], g[3]), p24 = vadd(g[2], g[4]);
    const T p56 = vadd(g[5], g[6]), p78 = vadd(g[7], g[8]);
    const T d58 = vadd(p56, p78);
    const T s10 = vadd(vadd(a13, a56), a87);
    const T s01 = vadd(vsub(g[2], g[4]), vsub(p56, p78));
    const T s20 = vadd(p13, d58);
    const T s02 = vadd(p24, d58);
    const T s11 = vsub(a56, a87);
    const T s00 = vadd(vadd(g[0], d58), vadd(p13, p24));

    // hydrodynamic fields (rho u = sum f e + F / (2 gamma))
    const T rho = vadd(splat<T>(1.0), s00);
    const T irho = vrcp(rho);
    const T jx = FORCE ? vadd(s10, k.hx) : s10;
    const T jy = FORCE ? vfma(k.r, s01, k.hy) : vmul(k.r, s01);
    const T ux = vmul(jx, irho), uy = vmul(jy, irho);
    const T ux2 = vmul(ux, ux), uy2 = vmul(uy, uy), uxy = vmul(ux, uy);
    const T rux2 = vmul(jx, ux), ruy2 = vmul(jy, uy), ruxy = vmul(jx, uy);
    const T sp = vadd(rux2, ruy2), sm = vsub(rux2, ruy2);
    const T c2s00 = vmul(k.c2, s00);

    // non-equilibrium central moments w.r.t. the base equilibria of Eq. 14
    T n2s = vfma(k.r2, s02, s20);
    n2s = vfma(splat<T>(-2.0), c2s00, n2s);
    n2s = vfma(k.nig, sp, n2s);
    T n2d = vfma(k.nr2, s02, s20);
    n2d = vfma(k.nig, sm, n2d);
    T n11 = vfma(k.r, s11, vmul(k.nig, ruxy));
    if (FORCE) {
        const T fx2 = vmul(ux, k.hx), fy2 = vmul(uy, k.hy);
        n2s = vfma(splat<T>(2.0), vadd(fx2, fy2), n2s);
        n2d = vfma(splat<T>(2.0), vsub(fx2, fy2), n2d);
        n11 = vfma(uy, k.hx, vfma(ux, k.hy, n11));
    }

    // The two unknowns X, Y of the strain-rate system (Eqs. 43-44) solve
    //   (Cb0 rho + a_x) X + (Cb0 rho + a_y) Y = R2s,
    //   (Cs0 rho + d_x) X + (n_y - Cs0 rho) Y = R2d,
    // with (P = P_gamma, Q = Q_gamma)
    //   a_x = rho (k3x + P u_x^2 / 2 + Q u_y^2 / 2),  a_y = rho (k3y + P u_y^2 / 2 + Q u_x^2 / 2),
    //   d_x = rho (k3x + P u_x^2 / 2 - Q u_y^2 / 2),  n_y = -rho (k3y + P u_y^2 / 2 - Q u_x^2 / 2).
    // The system is homogeneous in rho, and the moments below use X and Y
    // only as Xs = rho (X + Y) and Xd = rho (X - Y): by the two rows, the
    // corrections c_s = a_x X + a_y Y + nebr and c_d = d_x X + n_y Y + nesr
    // equal n2s - Cb0 Xs and n2d - Cs0 Xd.  So the system is solved for
    // (Xs, Xd) directly, with rho = 1 and its coefficients taken half:
    //   m11 = Cb0 + (k3x + k3y)/2 + (P + Q)/4 (u_x^2 + u_y^2),
    //   m12 = (k3x - k3y)/2 + (P - Q)/4 (u_x^2 - u_y^2),
    //   m21 = (k3x - k3y)/2 + (P + Q)/4 (u_x^2 - u_y^2),
    //   m22 = Cs0 + (k3x + k3y)/2 + (P - Q)/4 (u_x^2 + u_y^2).
    const T qp = vadd(ux2, uy2), qm = vsub(ux2, uy2);
    const T m11 = vfma(k.pp, qp, k.e1), m22 = vfma(k.pm, qp, k.e3);
    const T m12 = vfma(k.pm, qm, k.e2), nm21 = vfma(k.npp, qm, k.ne2);
    const T idet = vrcp(vfma(m11, m22, vmul(m12, nm21)));
    M = Moments<T>{s00, jx, jy, ux, uy, ux2, uy2, uxy, rux2, ruy2, ruxy, sp, sm, c2s00, n2s, n2d, n11,
                   m11, m22, m12, nm21, idet};
}

template <typename T, bool DRHO, bool FORCE, bool RAW = false>
PRC_HD void collide_relax(const Coef<T> &k, const Moments<T> &M, T g[9], T dxr, T dyr, T &ux_out, T &uy_out,
                          T &drho_out)
{
    const T s00 = M.s00, jx = M.jx, jy = M.jy, ux = M.ux, uy = M.uy;
    const T ux2 = M.ux2, uy2 = M.uy2, uxy = M.uxy, rux2 = M.rux2, ruy2 = M.ruy2, ruxy = M.ruxy;
    const T sp = M.sp, sm = M.sm, c2s00 = M.c2s00, n2s = M.n2s, n2d = M.n2d, n11 = M.n11;
    const T m11 = M.m11, m22 = M.m22, m12 = M.m12, nm21 = M.nm21, idet = M.idet;
    // local strain rates (Eqs. 43-48, R per Eq. 45); nebr = -e_b,rho, nesr = -e_s,rho
    T nebr = splat<T>(0.0), nesr = splat<T>(0.0);
    if (DRHO) {
        const T Adx = vmul(vmul(k.Ax, ux), dxr), Bdy = vmul(vmul(k.By, uy), dyr);
        nebr = vadd(Adx, Bdy);
        nesr = vsub(Adx, Bdy);
    }
    const T R2s = vsub(n2s, nebr), R2d = vsub(n2d, nesr);
    const T Xs = vmul(vsub(vmul(m22, R2s), vmul(m12, R2d)), idet);
    const T Xd = vmul(vfma(m11, R2d, vmul(nm21, R2s)), idet);

    // extended-equilibrium corrections (Eqs. 30, 38-40 / App. A) and
    // relaxation.  Relaxing n2s at omega_xi and adding -omega_xi tau_xi times
    // its correction n2s - Cb0 Xs leaves -n2s / 2 + omega_xi tau_xi Cb0 Xs
    // ((1 - omega)/2 - omega tau = -1/2); likewise for n2d.
    // b20 = c^2 s00 + (k~2s - 2 c^2 rho)/2, ht2d = k~2d / 2, t11x2 = 2 k~11
    T b20 = vfma(k.hh1, sp, vfma(splat<T>(-0.5), n2s, vfma(k.kS, Xs, c2s00)));
    T ht2d = vfma(k.hh1, sm, vfma(splat<T>(-0.5), n2d, vmul(k.kD, Xd)));
    T t11x2 = vfma(k.h1x2, ruxy, vfma(k.omw2, n11, vmul(vmul(k.kdQg2, uxy), Xs)));
    if (DRHO) t11x2 = vfma(k.kdh1c2x2, vfma(uy, dxr, vmul(ux, dyr)), t11x2);
    if (FORCE) {
        b20 = vfma(k.fsx, ux, vfma(k.fsy, uy, b20));
        ht2d = vfma(k.fdx, ux, vfma(k.nfdy, uy, ht2d));
        t11x2 = vfma(k.fdx2, uy, vfma(k.fdy2, ux, t11x2));
    }
    const T E20 = vadd(b20, ht2d), E02 = vsub(b20, ht2d);  // c^2 s00 + k~20 - c^2 rho, and for 02
    const T t20 = vadd(E20, k.c2), t02 = vadd(E02, k.c2);   // k~20, k~02 (c^2 rho = c^2 + c^2 s00)

    // post-collision raw moments minus the rest-state moments (F^-1), with
    // k~21 = a3 rho u_x^2 u_y, k~12 = a3 rho u_x u_y^2, k~22 = c^4 rho
    const T e21 = vmul(rux2, uy), e12 = vmul(ruy2, ux);
    T D10 = jx, D01 = jy;
    T D20 = vadd(E20, rux2);
    T D02 = vadd(E02, ruy2);
    T D11 = vfma(splat<T>(0.5), t11x2, ruxy);
    T D21, D12, D22;
    if constexpr (RAW) {
        // raw equilibria of Eq. 12: rho (c^2 + u_x^2 / g^2) u_y, rho (c^2 +
        // u_y^2 / g^2) u_x, rho c^4 + rho c^2 (u_x^2 + u_y^2) + rho u_x^2 u_y^2
        D21 = vfma(k.c2, jy, vmul(k.ig2, e21));
        D12 = vfma(k.c2, jx, vmul(k.ig2, e12));
        D22 = vfma(k.c4, s00, vfma(k.c2, sp, vmul(e21, uy)));
    } else {
        D21 = vfma(k.a3p1, e21, vfma(ux, t11x2, vmul(uy, t20)));
        D12 = vfma(k.a3p1, e12, vfma(uy, t11x2, vmul(ux, t02)));
        D22 = vfma(ux2, t02, vfma(uy2, t20, vfma(vadd(uxy, uxy), t11x2,
                                                 vfma(k.a34p1, vmul(e21, uy), vmul(k.c4, s00)))));
    }
    if (FORCE) {
        const T hxuy = vmul(k.hx, uy), hyux = vmul(k.hy, ux);
        D10 = vadd(D10, k.hx);
        D01 = vadd(D01, k.hy);
        D20 = vfma(vadd(ux, ux), k.hx, D20);
        D02 = vfma(vadd(uy, uy), k.hy, D02);
        D11 = vadd(D11, vadd(hxuy, hyux));
        if constexpr (!RAW) {
            D21 = vfma(ux, vfma(splat<T>(2.0), hxuy, hyux), D21);
            D12 = vfma(uy, vfma(splat<T>(2.0), hyux, hxuy), D12);
            D22 = vfma(vadd(uxy, uxy), vadd(hxuy, hyux), D22);
        }
    }

    // S^-1 then P^-1 (Eq. 72) with the 1/2, 1/4 and 1/r^n factors folded
    // (Z21, Z12 = -2 Q21, -2 Q12 exactly: the scalings differ by a power of two)
    const T Q11 = vmul(D11, k.qr), Q22 = vmul(D22, k.qr2), Z21 = vmul(D21, k.n2qr), Z12 = vmul(D12, k.n2qr2);
    const T p = vfma(splat<T>(-0.5), Z21, Q22), m = vfma(splat<T>(-0.5), Z12, Q11);
    const T pp = vfma(splat<T>(0.5), Z21, Q22), mm = vfma(splat<T>(0.5), Z12, Q11);
    g[5] = vadd(p, m);
    g[6] = vsub(p, m);
    g[7] = vadd(pp, mm);
    g[8] = vsub(pp, mm);
    const T n2Q22 = vmul(splat<T>(-2.0), Q22);
    const T a1 = vfma(splat<T>(0.5), D20, n2Q22);
    const T b1 = vfma(splat<T>(0.5), D10, Z12);
    g[1] = vadd(a1, b1);
    g[3] = vsub(a1, b1);
    const T a2 = vfma(k.hr2, D02, n2Q22);
    const T b2 = vfma(k.hr, D01, Z21);
    g[2] = vadd(a2, b2);
    g[4] = vsub(a2, b2);
    g[0] = vfma(splat<T>(4.0), Q22, vfma(k.ninv_r2, D02, vsub(s00, D20)));

    ux_out = ux;
    uy_out = uy;
    drho_out = s00;
}

template <typename T, bool DRHO, bool FORCE, bool RAW = false>
PRC_HD void collide(const Coef<T> &k, T g[9], T dxr, T dyr, T &ux_out, T &uy_out, T &drho_out)
{
    Moments<T> M;
    collide_moments<T, FORCE>(k, g, M);
    collide_relax<T, DRHO, FORCE, RAW>(k, M, g, dxr, dyr, ux_out, uy_out, drho_out);
}

}  // namespace prc
