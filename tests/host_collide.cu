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
