// host_collide.cu -- test harness, not part of the library: the collision of
// prc_device.cuh (the code the GPU kernels run) built for the host, so that
// tests/test_host_collision.py can compare its FP64 arithmetic with the
// oracle's matrix form node by node without a GPU.  The coefficients come from
// the library's own host set-up (prc_host.h).
#include <cstring>

#include "prc_host.h"

namespace {

template <bool DRHO, bool FORCE, bool RAW>
void run(const prc::Coef<double> &k, double *g, double dxr, double dyr, double *diag)
{
    double ux = 0.0, uy = 0.0, drho = 0.0;
    prc::collide<double, DRHO, FORCE, RAW>(k, g, dxr, dyr, ux, uy, drho);
    diag[0] = ux;
    diag[1] = uy;
    diag[2] = drho;
}

template <bool RAW>
void dispatch(const prc::Coef<double> &k, bool drho, bool force, double *g, double dxr, double dyr, double *diag)
{
    if (drho) {
        if (force) run<true, true, RAW>(k, g, dxr, dyr, diag);
        else run<true, false, RAW>(k, g, dxr, dyr, diag);
    } else {
        if (force) run<false, true, RAW>(k, g, dxr, dyr, diag);
        else run<false, false, RAW>(k, g, dxr, dyr, diag);
    }
}

}  // namespace

// One collision of the shifted populations g_in (f - w) of a node with
// density gradient (dxr, dyr); g_out the post-collision shifted populations,
// w_out the library's rest populations w_i(r), diag (u_x, u_y, rho - 1).
extern "C" int host_collide(double r, double gamma, double nu, double omega_xi, double fx, double fy, int drho,
                            int model, const double *g_in, double dxr, double dyr, double *g_out, double *w_out,
                            double *diag)
{
    lbm_params p;
    std::memset(&p, 0, sizeof p);
    p.nx = 8;
    p.ny = 8;
    p.r = r;
    p.gamma = gamma;
    p.nu = nu;
    p.omega_xi = omega_xi;
    p.fx = fx;
    p.fy = fy;
    p.dtype = LBM_F64;
    p.bc = LBM_BC_CAVITY;
    p.drho = drho ? LBM_DRHO_CURRENT : LBM_DRHO_OFF;
    p.model = model;
    prc::Coef<double> k;
    prc_host::make_coef(p, k);
    for (int i = 0; i < 9; i++) {
        g_out[i] = g_in[i];
        w_out[i] = k.w[i];
    }
    const bool force = fx != 0.0 || fy != 0.0;
    if (model == LBM_MODEL_PRNR) dispatch<true>(k, drho != 0, force, g_out, dxr, dyr, diag);
    else dispatch<false>(k, drho != 0, force, g_out, dxr, dyr, diag);
    return 0;
}

// The FP32 collision of two nodes a, b: packed as the lanes of one F2 (as the
// FP32 / FP16 kernels run it) and each alone as float.  g_ab holds node a's
// nine shifted populations then node b's; out_pair and out_single receive the
// post-collision populations in the same order.
extern "C" int host_collide_f32_pair(double r, double gamma, double nu, double omega_xi, int model,
                                     const double *g_ab, const double *dx_ab, const double *dy_ab,
                                     float *out_pair, float *out_single)
{
    lbm_params p;
    std::memset(&p, 0, sizeof p);
    p.nx = 8;
    p.ny = 8;
    p.r = r;
    p.gamma = gamma;
    p.nu = nu;
    p.omega_xi = omega_xi;
    p.dtype = LBM_F32;
    p.bc = LBM_BC_CAVITY;
    p.drho = LBM_DRHO_CURRENT;
    p.model = model;
    prc::Coef<double> kd;
    prc_host::make_coef(p, kd);
    prc::Coef<float> kf;
    prc::Coef<prc::F2> k2;
    const double *s = reinterpret_cast<const double *>(&kd);
    float *of = reinterpret_cast<float *>(&kf);
    prc::F2 *o2 = reinterpret_cast<prc::F2 *>(&k2);
    for (size_t i = 0; i < sizeof(kd) / sizeof(double); i++) {
        of[i] = (float)s[i];
        o2[i] = prc::F2((float)s[i]);
    }
    prc::F2 g2[9];
    for (int i = 0; i < 9; i++) g2[i] = prc::F2((float)g_ab[i], (float)g_ab[9 + i]);
    prc::F2 ux2, uy2, d2;
    const prc::F2 dx2((float)dx_ab[0], (float)dx_ab[1]), dy2((float)dy_ab[0], (float)dy_ab[1]);
    if (model == LBM_MODEL_PRNR) prc::collide<prc::F2, true, false, true>(k2, g2, dx2, dy2, ux2, uy2, d2);
    else prc::collide<prc::F2, true, false, false>(k2, g2, dx2, dy2, ux2, uy2, d2);
    for (int i = 0; i < 9; i++) {
        out_pair[i] = g2[i].v.x;
        out_pair[9 + i] = g2[i].v.y;
    }
    for (int n = 0; n < 2; n++) {
        float g1[9], ux, uy, d;
        for (int i = 0; i < 9; i++) g1[i] = (float)g_ab[9 * n + i];
        if (model == LBM_MODEL_PRNR)
            prc::collide<float, true, false, true>(kf, g1, (float)dx_ab[n], (float)dy_ab[n], ux, uy, d);
        else prc::collide<float, true, false, false>(kf, g1, (float)dx_ab[n], (float)dy_ab[n], ux, uy, d);
        for (int i = 0; i < 9; i++) out_single[9 * n + i] = g1[i];
    }
    return 0;
}
