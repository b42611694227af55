// prc_host.h -- host-side helpers shared by the single-instance and batch C
// ABIs: per-instance constants, storage layout, launch plan.  Internal.
#pragma once

#include <cmath>
#include <cstring>

#include "prc_lbm.h"
#include "prc_ops.h"

namespace prc_host {

using prc::Coef;
using prc::DevStatus;
using prc::Grid;
using prc::Plan;

constexpr size_t ALIGN = 256;

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline const prc::DtypeOps *ops_for(int dtype)
{
    switch (dtype) {
    case LBM_F64: return &prc::ops_f64;
    case LBM_F32: return &prc::ops_f32;
    case LBM_F16: return &prc::ops_f16;
    default: return nullptr;
    }
}

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

inline void add_rect(prc::Rects &rc, int x0, int y0, int x1, int y1, int lw, int threads)
{
    if (x1 <= x0 || y1 <= y0) return;
    const int i = rc.n++;
    rc.x0[i] = x0;
    rc.y0[i] = y0;
    rc.x1[i] = x1;
    rc.y1[i] = y1;
    rc.lw[i] = lw;
    rc.tiles_x[i] = ceil_div(x1 - x0, 1 << lw);
    rc.start[i + 1] = rc.start[i] + rc.tiles_x[i] * ceil_div(y1 - y0, threads >> lw);
}

// Tile width (log2) for a w x h strip covered by CTAs of `threads` threads:
// the fewest tiles, then the widest (coalesced rows).
inline int strip_lw(int w, int h, int threads)
{
    int best = 1;
    long long best_tiles = -1;
    for (int lw = 1; (2 << lw) <= threads; lw++) {
        const long long t = (long long)ceil_div(w, 1 << lw) * ceil_div(h, threads >> lw);
        if (best_tiles < 0 || t <= best_tiles) {
            best = lw;
            best_tiles = t;
        }
    }
    return best;
}

inline void add_strip(prc::Rects &rc, int x0, int y0, int x1, int y1, int threads)
{
    add_rect(rc, x0, y0, x1, y1, strip_lw(x1 - x0, y1 - y0, threads), threads);
}

// Split of one step between the TMA interior kernel (tiles at least two nodes
// from every wall, x origin 16-byte aligned) and the general tile body on the
// remaining edge strips.  With the interior kernel, the strips are covered by
// the same launch after its interior tiles (tile shapes fitted to the strips);
// otherwise the general kernel covers the whole domain in 32 x 8 tiles.
// num_sms <= 0 gives the upper bound used to size the workspace.
inline Plan make_plan(const lbm_params &p, int num_sms, int variant)
{
    const prc::DtypeOps *ops = ops_for(p.dtype);
    Plan pl;
    std::memset(&pl, 0, sizeof(pl));
    const bool have = variant >= 0 && variant < ops->nvariants;
    const int W = have ? ops->variants[variant].w : 0, H = have ? ops->variants[variant].h : 0;
    const int PX = ops->tma_padx;
    const int ix0 = PX, iy0 = 2;
    // the interior kernel implements the central scheme only
    if (have && p.model == LBM_MODEL_PRC && p.nx - 2 - ix0 >= W && p.ny - 2 - iy0 >= H) {
        const int threads = ops->variants[variant].threads;
        const int xlast = ((p.nx - 2 - W) / PX) * PX;
        const int ylast = p.ny - 2 - H;
        const int xend = xlast + W, yend = ylast + H;
        pl.tma = 1;
        pl.in.ix0 = ix0;
        pl.in.iy0 = iy0;
        pl.in.ntx = ceil_div(xend - ix0, W);
        pl.in.nty = ceil_div(yend - iy0, H);
        pl.in.xlast = xlast;
        pl.in.ylast = ylast;
        const int ntiles = pl.in.ntx * pl.in.nty;
        int g = ntiles < prc::MAX_INTERIOR_CTAS ? ntiles : prc::MAX_INTERIOR_CTAS;
        const int resident = num_sms * ops->variants[variant].ctas_per_sm;
        if (num_sms > 0 && g > resident) g = resident;
        pl.n_int_ctas = g;
        add_strip(pl.edge, 0, 0, p.nx, iy0, threads);
        add_strip(pl.edge, 0, yend, p.nx, p.ny, threads);
        add_strip(pl.edge, 0, iy0, ix0, yend, threads);
        add_strip(pl.edge, xend, iy0, p.nx, yend, threads);
        pl.n_edge_ctas = 0;  // the strips ride in the interior launch
    } else {
        // general kernel over the whole grid: 32 x 8 tiles of one node per
        // thread (FP64), 64 x 8 tiles of node pairs (FP32 collision)
        if (p.dtype == LBM_F64) add_rect(pl.edge, 0, 0, p.nx, p.ny, 5, prc::BX * prc::BY);
        else add_rect(pl.edge, 0, 0, p.nx, p.ny, 6, prc::PTW * prc::PTH);  // 2^6 x (512 >> 6) nodes
        pl.n_edge_ctas = pl.edge.start[pl.edge.n];
    }
    pl.nparts = pl.n_int_ctas + pl.n_edge_ctas;
    return pl;
}

// cuTensorMapEncodeTiled, looked up once through the runtime's driver entry
// points (null when unavailable).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn tensor_map_encoder()
{
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess) return nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// 3-D tiled descriptor over one population set, (x < nx, y < ny, plane < 9),
// with a box of bw x bh x 1 elements of `elem` bytes.
inline CUresult encode_pop_map(CUtensorMap *m, size_t elem, void *base, int nx, int ny, int pitch, size_t plane, int bw,
                               int bh, CUtensorMapL2promotion l2)
{
    const EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return CUDA_ERROR_NOT_SUPPORTED;
    const CUtensorMapDataType dt = elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : (elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * elem, (cuuint64_t)plane * elem};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, l2,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

struct Layout {
    int pitch;
    size_t plane, pop_bytes, snap_bytes, part_bytes, st_bytes;
    size_t off_pop0, off_pop1, off_snap, off_part, off_st, total;
    int nparts;
};

inline Layout make_layout(const lbm_params &p)
{
    const prc::DtypeOps *ops = ops_for(p.dtype);
    Layout L;
    L.pitch = (int)align_up((size_t)p.nx, 32);
    L.plane = (size_t)L.pitch * (size_t)p.ny;
    L.pop_bytes = align_up(9 * L.plane * ops->elem, ALIGN);
    L.snap_bytes = align_up(L.plane * ops->snap_elem, ALIGN);
    int np = ((p.nx + 31) / 32) * ((p.ny + 7) / 8);  // mass reduction
    for (int v = -1; v < ops->nvariants; v++) {
        const int n = make_plan(p, 0, v).nparts;
        if (n > np) np = n;
    }
    L.nparts = np;
    L.part_bytes = align_up((size_t)L.nparts * sizeof(double2), ALIGN);
    L.st_bytes = align_up(sizeof(DevStatus), ALIGN);
    L.off_pop0 = 0;
    L.off_pop1 = L.off_pop0 + L.pop_bytes;
    L.off_snap = L.off_pop1 + L.pop_bytes;
    L.off_part = L.off_snap + L.snap_bytes;
    L.off_st = L.off_part + L.part_bytes;
    L.total = L.off_st + L.st_bytes;
    return L;
}

inline double q_of(double r) { return r < 1.0 ? r : 1.0; }

inline double omega_nu_of(const lbm_params &p)
{
    const double c2 = q_of(p.r) * q_of(p.r) / 3.0;
    return 1.0 / (p.nu / (p.gamma * c2) + 0.5);
}

// Per-instance constants (App. A coefficients with dt = 1), in the folded
// form the device collision uses.
inline void make_coef(const lbm_params &p, Coef<double> &k)
{
    std::memset(&k, 0, sizeof(k));
    const double r = p.r, q = q_of(r), c2 = q * q / 3.0, g = p.gamma;
    const double w_nu = omega_nu_of(p), w_xi = p.omega_xi;
    const double tau_nu = 1.0 / w_nu - 0.5, tau_xi = 1.0 / w_xi - 0.5;
    const double Pg = 4.0 / (g * g) - 1.0 / g, Qg = 1.0 / (g * g) - 1.0 / g, Ug = 2.0 / g + 1.0;
    const double a3 = 1.0 / (g * g) - 3.0 / g + 2.0;
    const double k3x = 0.5 * (3.0 * c2 - 1.0), k3y = 0.5 * (3.0 * c2 - r * r);
    const double Cb0 = -2.0 * c2 / w_xi, Cs0 = -2.0 * c2 / w_nu;
    const double kd = -w_nu * tau_nu, kxs = -w_xi * tau_xi;
    const double fdx = (1.0 - 0.5 * w_nu) * Qg * p.fx, fdy = (1.0 - 0.5 * w_nu) * Qg * p.fy;
    k.r = r;
    k.r2 = r * r;
    k.c2 = c2;
    k.c4 = c2 * c2;
    k.hh1 = 0.5 * (1.0 / g - 1.0);
    k.Ax = 0.5 * (Ug * c2 - 1.0);
    k.By = 0.5 * (Ug * c2 - r * r);
    k.pp = 0.25 * (Pg + Qg);
    k.npp = -k.pp;
    k.pm = 0.25 * (Pg - Qg);
    k.e1 = Cb0 + 0.5 * (k3x + k3y);
    k.e2 = 0.5 * (k3x - k3y);
    k.ne2 = -k.e2;
    k.e3 = Cs0 + 0.5 * (k3x + k3y);
    k.kS = -kxs * Cb0;
    k.kD = -kd * Cs0;
    k.h1x2 = 2.0 * (1.0 / g - 1.0);
    k.omw2 = 2.0 * (1.0 - w_nu);
    k.kdQg2 = 2.0 * kd * Qg;
    k.kdh1c2x2 = 2.0 * kd * (1.0 / g - 1.0) * c2;
    k.a3p1 = a3 + 1.0;
    k.a34p1 = 4.0 * a3 + 1.0;
    k.qr = 0.25 / r;
    k.qr2 = 0.25 / (r * r);
    k.hr = 0.5 / r;
    k.hr2 = 0.5 / (r * r);
    k.inv_r2 = 1.0 / (r * r);
    k.n2qr = -2.0 * k.qr;
    k.n2qr2 = -2.0 * k.qr2;
    k.hx = p.fx / (2.0 * g);
    k.hy = p.fy / (2.0 * g);
    k.fsx = (1.0 - 0.5 * w_xi) * Qg * p.fx;
    k.fsy = (1.0 - 0.5 * w_xi) * Qg * p.fy;
    k.fdx = fdx;
    k.nfdy = -fdy;
    k.fdx2 = 2.0 * fdx;
    k.fdy2 = 2.0 * fdy;
    k.nig = -1.0 / g;
    k.nr2 = -k.r2;
    k.ninv_r2 = -k.inv_r2;
    const bool lid_on = (p.bc != LBM_BC_PERIODIC) && (p.u_lid != 0.0);
    k.lid = lid_on ? c2 * p.u_lid / (2.0 * r * r) : 0.0;
    k.ig2 = 1.0 / (g * g);
    k.inv12 = 1.0 / 12.0;
    k.inv12r = 1.0 / (12.0 * r);
    // rest populations: the unique f with the rest moments (1, 0, 0, c^2,
    // c^2, 0, 0, 0, c^4) of Eq. 12 at u = 0, through S^-1 and P^-1
    const double a = c2, b = c2 / (r * r), cc = c2 * c2 / (r * r);
    k.w[0] = 1.0 - a - b + cc;
    k.w[1] = k.w[3] = 0.5 * (a - cc);
    k.w[2] = k.w[4] = 0.5 * (b - cc);
    k.w[5] = k.w[6] = k.w[7] = k.w[8] = 0.25 * cc;
}

inline Grid make_grid(const lbm_params &p, const Layout &L)
{
    Grid gd;
    gd.nx = p.nx;
    gd.ny = p.ny;
    gd.pitch = L.pitch;
    gd.bc = p.bc;
    gd.plane = (long long)L.plane;
    gd.lid_on = (p.bc != LBM_BC_PERIODIC) && (p.u_lid != 0.0);
    gd.model = p.model;
    return gd;
}

}  // namespace prc_host
