// lbm_api.cu -- the C ABI of include/prc_lbm.h: handles, workspace layout,
// per-instance constants, step scheduling (CUDA graphs of 20 steps), the
// device-side stop rule of lbm_run, residual/mass finalisation, field and
// population transfers, checkpoints.
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <cuda.h>

#include "prc_host.h"
#include "prc_lbm.h"
#include "prc_ops.h"

using prc::Coef;
using prc::DevStatus;
using prc::Grid;
using prc::Plan;
using namespace prc_host;

namespace {

constexpr int RES_INTERVAL = 20;  // residual every 20 steps (Sec. 5.2)

thread_local std::string g_err;

// Fixed-order two-level reduction of the per-CTA partials (deterministic).
__device__ void reduce_partials(const double2 *partials, int n, double &a, double &b)
{
    __shared__ double sa[256], sb[256];
    const int t = threadIdx.x;
    double x = 0.0, y = 0.0;
    for (int i = t; i < n; i += 256) {
        x += partials[i].x;
        y += partials[i].y;
    }
    sa[t] = x;
    sb[t] = y;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) {
            sa[t] += sa[t + s];
            sb[t] += sb[t + s];
        }
        __syncthreads();
    }
    a = sa[0];
    b = sb[0];
}

// Residual and mass of a residual step; the stop rule of lbm_run.
__global__ void __launch_bounds__(256) k_finalize(const double2 *partials, int n, DevStatus *st, double nnodes)
{
    if (st->stop) return;
    double a, b;
    reduce_partials(partials, n, a, b);
    if (threadIdx.x == 0) {
        const double res = sqrt(a), mass = nnodes + b;
        st->res_step += RES_INTERVAL;
        st->res = res;
        st->mass = mass;
        if (!isfinite(res) || !isfinite(mass)) {
            st->diverged = 1;
            st->stop = 1;
        } else if (res < st->tol) {
            st->converged = 1;
            st->stop = 1;
        }
    }
}

__global__ void __launch_bounds__(256) k_mass_final(const double2 *partials, int n, DevStatus *st, double nnodes)
{
    double a, b;
    reduce_partials(partials, n, a, b);
    if (threadIdx.x == 0) st->mass_now = nnodes + b;
}

__global__ void k_status_reset(DevStatus *st)
{
    st->stop = 0;
    st->converged = 0;
    st->diverged = 0;
    st->timeout = 0;
    st->res_step = 0;
    st->tol = -1.0;
    st->res = INFINITY;
    st->mass = 0.0;
    st->mass_now = 0.0;
}

__global__ void k_status_arm(DevStatus *st, double tol)
{
    st->tol = tol;
    st->converged = 0;
    st->stop = st->diverged ? 1 : 0;
}

}  // namespace

struct lbm_s {
    lbm_params p;
    const prc::DtypeOps *ops;
    Layout L;
    Grid gd;
    Coef<double> k;
    int device;
    cudaStream_t stream;
    bool own_stream;
    char *ws;
    bool own_ws;
    void *pop[2];
    void *snap;
    double2 *partials;
    DevStatus *st;
    DevStatus *st_host;  // pinned mirror
    long long t;         // completed steps; invariant: the state is in pop[t & 1]
    Plan plan;
    int variant;          // interior-kernel variant (-1: general kernel only)
    int num_sms;
    CUtensorMap tmap[2];     // TMA load descriptors of the two population sets (box = tile + ring)
    CUtensorMap tmap_st[2];  // TMA store descriptors of the two sets (box = tile)
    prc::ClusterGeom cgeo;  // cluster-resident engine (variant LBM_VARIANT_CLUSTER)
    cudaGraphExec_t g20;
    bool have_g20;
    std::string err;
};

namespace {

lbm_status fail(lbm_t h, lbm_status s, const std::string &msg)
{
    if (h) h->err = msg;
    else g_err = msg;
    return s;
}

lbm_status cuda_fail(lbm_t h, cudaError_t e, const char *what)
{
    return fail(h, LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                          \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

lbm_status enter(lbm_t h)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "null handle");
    h->err.clear();
    CK(h, cudaSetDevice(h->device));
    return LBM_OK;
}

void *cur_pop(lbm_t h) { return h->pop[h->t & 1]; }

bool is_cluster(lbm_t h) { return h->variant == LBM_VARIANT_CLUSTER; }

// n steps of the cluster-resident engine in one launch (state after step
// t_before in pop[t_before & 1])
lbm_status launch_cluster(lbm_t h, cudaStream_t s, long long t_before, long long n)
{
    const bool drho = h->p.drho == LBM_DRHO_CURRENT, force = h->p.fx != 0.0 || h->p.fy != 0.0;
    CK(h, h->ops->cluster_launch(h->pop[0], h->pop[1], h->gd, h->k, h->snap, h->st, t_before, (int)n, h->cgeo.nc,
                                 h->cgeo.rpc, h->cgeo.smem, drho, force, s));
    return LBM_OK;
}

// one step; the state moves from pop[t&1] to pop[(t+1)&1]
lbm_status launch_one(lbm_t h, cudaStream_t s, long long t_before)
{
    if (is_cluster(h)) return launch_cluster(h, s, t_before, 1);
    const bool epi = ((t_before + 1) % RES_INTERVAL) == 0;
    const int c = (int)(t_before & 1);
    const bool drho = h->p.drho == LBM_DRHO_CURRENT, force = h->p.fx != 0.0 || h->p.fy != 0.0;
    if (h->plan.tma)
        CK(h, h->ops->variants[h->variant].launch(&h->tmap[c], &h->tmap_st[c ^ 1], h->pop[c], h->pop[c ^ 1], h->plan,
                                                   h->gd, h->k, h->snap, h->partials, h->st, drho, epi, force, c, s));
    if (h->plan.n_edge_ctas > 0)
        CK(h, h->ops->step_general(h->pop[c], h->pop[c ^ 1], h->plan, h->gd, h->k, h->snap, h->partials, h->st,
                                   drho, epi, force, s));
    if (epi) {
        k_finalize<<<1, 256, 0, s>>>(h->partials, h->plan.nparts, h->st, (double)h->p.nx * (double)h->p.ny);
        CK(h, cudaGetLastError());
    }
    return LBM_OK;
}

// CUDA graph of the 20 steps t = 20m .. 20m+19 (state starts and ends in pop[0]).
lbm_status ensure_graph(lbm_t h)
{
    if (h->have_g20) return LBM_OK;
    cudaStream_t cs;
    CK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_fail(h, e, "cudaStreamBeginCapture");
    }
    lbm_status st = LBM_OK;
    for (int i = 0; i < RES_INTERVAL && st == LBM_OK; i++) st = launch_one(h, cs, i);
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (st != LBM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->g20, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    h->have_g20 = true;
    return LBM_OK;
}

lbm_status enqueue_steps(lbm_t h, long long n)
{
    if (is_cluster(h)) {
        while (n > 0) {  // the device steps in one launch per chunk; no graph needed
            const long long c = n < (1LL << 30) ? n : (1LL << 30);
            lbm_status s = launch_cluster(h, h->stream, h->t, c);
            if (s != LBM_OK) return s;
            h->t += c;
            n -= c;
        }
        return LBM_OK;
    }
    while (n > 0) {
        if ((h->t % RES_INTERVAL) == 0 && n >= RES_INTERVAL) {
            lbm_status s = ensure_graph(h);
            if (s != LBM_OK) return s;
            CK(h, cudaGraphLaunch(h->g20, h->stream));
            h->t += RES_INTERVAL;
            n -= RES_INTERVAL;
        } else {
            lbm_status s = launch_one(h, h->stream, h->t);
            if (s != LBM_OK) return s;
            h->t += 1;
            n -= 1;
        }
    }
    return LBM_OK;
}

lbm_status read_status(lbm_t h)
{
    CK(h, cudaMemcpyAsync(h->st_host, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status reset_state_meta(lbm_t h)
{
    h->t = 0;
    k_status_reset<<<1, 1, 0, h->stream>>>(h->st);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

// device scratch for host<->device transfers of fields / populations
struct DevTmp {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~DevTmp()
    {
        if (p) cudaFreeAsync(p, s);
    }
};

// 3-D tiled descriptors over one population set: (x < nx, y < ny, plane < 9).
// Load: box = interior tile + ring, x widened to 16-byte aligned edges.
// Store: box = interior tile (its x origin is 16-byte aligned, and it lies
// inside the grid, so no store starts at a negative coordinate).
lbm_status make_tmaps(lbm_t h)
{
    if (!tensor_map_encoder()) return fail(h, LBM_ECUDA, "cuTensorMapEncodeTiled not available");
    const size_t elem = h->ops->elem;
    const prc::Variant &v = h->ops->variants[h->variant];
    for (int b = 0; b < 2; b++) {
        CUresult r = encode_pop_map(&h->tmap[b], elem, h->pop[b], h->p.nx, h->p.ny, h->L.pitch, h->L.plane,
                                    v.w + 2 * h->ops->tma_padx, v.h + 2, CU_TENSOR_MAP_L2_PROMOTION_L2_256B);
        if (r != CUDA_SUCCESS) return fail(h, LBM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        r = encode_pop_map(&h->tmap_st[b], elem, h->pop[b], h->p.nx, h->p.ny, h->L.pitch, h->L.plane, v.w, v.h,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE);
        if (r != CUDA_SUCCESS) return fail(h, LBM_ECUDA, "cuTensorMapEncodeTiled (store) failed (" + std::to_string((int)r) + ")");
    }
    return LBM_OK;
}

// Select the interior-kernel variant (-1: general kernel everywhere): plan,
// TMA descriptors, shared-memory opt-in; drops the captured graph.
// Geometry of the cluster-resident engine for h's grid: the largest cluster
// (at most 16 CTAs, one slab of >= 2 rows each) whose slabs fit the shared
// memory of a CTA and which the device can launch.
lbm_status cluster_select(lbm_t h, prc::ClusterGeom &g)
{
    int optin = 0;
    CK(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const int budget = optin - 1024;  // static shared memory of the kernel
    // The opt-in limit is an attribute of the kernel, shared by every handle
    // in the process: it is set to the whole budget (the same value from any
    // handle), never to this grid's size, which would make the launches of an
    // earlier handle with larger slabs fail.
    CK(h, h->ops->cluster_prepare(budget));
    for (int nc = prc::CL_MAX_CTAS; nc >= 1; nc--) {
        const int rpc = (h->p.ny + nc - 1) / nc;
        const int last = h->p.ny - (nc - 1) * rpc;
        if (rpc < 2 || last < 2) continue;
        const size_t smem = prc::cluster_smem_bytes(rpc, h->p.nx, h->ops->elem, h->ops->snap_elem);
        if (smem > (size_t)budget) continue;
        int active = 0;
        if (h->ops->cluster_max_active(nc, (int)smem, &active) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (active < 1) continue;
        g.nc = nc;
        g.rpc = rpc;
        g.smem = (int)smem;
        return LBM_OK;
    }
    return fail(h, LBM_EINVAL, "grid too large for the cluster-resident engine");
}

lbm_status apply_variant(lbm_t h, int variant)
{
    if (variant == LBM_VARIANT_CLUSTER) {
        prc::ClusterGeom g;
        lbm_status cs = cluster_select(h, g);
        if (cs != LBM_OK) return cs;
        h->cgeo = g;
        h->variant = variant;
        h->plan = make_plan(h->p, h->num_sms, -1);  // unused by the engine; kept consistent
        if (h->have_g20) {
            cudaGraphExecDestroy(h->g20);
            h->have_g20 = false;
        }
        return LBM_OK;
    }
    if (variant < -1 || variant >= h->ops->nvariants) return fail(h, LBM_EINVAL, "no such variant");
    if (variant >= 0 && h->p.model != LBM_MODEL_PRC)
        return fail(h, LBM_EINVAL, "the interior kernel implements the central scheme only");
    h->variant = variant;
    h->plan = make_plan(h->p, h->num_sms, variant);
    if (h->plan.tma) {
        lbm_status ts = make_tmaps(h);
        if (ts != LBM_OK) return ts;
        CK(h, h->ops->variants[variant].prepare());
    }
    if (h->have_g20) {
        cudaGraphExecDestroy(h->g20);
        h->have_g20 = false;
    }
    return LBM_OK;
}

lbm_status init_handle(lbm_t h, const lbm_params &p, void *ws, size_t ws_bytes, bool own_ws, cudaStream_t stream,
                       bool own_stream)
{
    h->p = p;
    h->ops = ops_for(p.dtype);
    h->L = make_layout(p);
    h->gd = make_grid(p, h->L);
    make_coef(p, h->k);
    h->stream = stream;
    h->own_stream = own_stream;
    h->ws = static_cast<char *>(ws);
    h->own_ws = own_ws;
    (void)ws_bytes;
    h->pop[0] = h->ws + h->L.off_pop0;
    h->pop[1] = h->ws + h->L.off_pop1;
    h->snap = h->ws + h->L.off_snap;
    h->partials = reinterpret_cast<double2 *>(h->ws + h->L.off_part);
    h->st = reinterpret_cast<DevStatus *>(h->ws + h->L.off_st);
    h->t = 0;
    h->have_g20 = false;
    CK(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    // small grids: the cluster-resident engine; otherwise the first interior
    // variant (or the general kernel when none is compiled)
    lbm_status vs = apply_variant(h, LBM_VARIANT_CLUSTER);
    if (vs != LBM_OK) {
        h->err.clear();
        vs = apply_variant(h, h->ops->nvariants > 0 && p.model == LBM_MODEL_PRC ? 0 : -1);
    }
    if (vs != LBM_OK) return vs;
    CK(h, cudaMallocHost(&h->st_host, sizeof(DevStatus)));
    // rest state f~ = w(r): zero shifted storage everywhere (padding too);
    // the residual snapshot holds its u_x (-F/(2 gamma) under a body force)
    CK(h, cudaMemsetAsync(h->ws, 0, h->L.off_part, h->stream));
    CK(h, h->ops->fields(h->pop[0], h->gd, h->k, nullptr, nullptr, nullptr, h->snap, h->stream));
    return reset_state_meta(h);
}

}  // namespace

// ---------------------------------------------------------------------------
// public entry points

extern "C" {

lbm_status lbm_params_init(lbm_params *p, int nx, int ny, double r, double gamma, double nu, double u_lid,
                           int dtype)
{
    if (!p) return fail(nullptr, LBM_EINVAL, "null params");
    std::memset(p, 0, sizeof(*p));
    p->nx = nx;
    p->ny = ny;
    p->r = r;
    p->gamma = gamma;
    p->nu = nu;
    p->u_lid = u_lid;
    p->omega_xi = 1.0;
    p->dtype = dtype;
    p->bc = LBM_BC_CAVITY;
    p->drho = LBM_DRHO_CURRENT;
    p->model = LBM_MODEL_PRC;
    return LBM_OK;
}

lbm_status lbm_params_check(const lbm_params *p)
{
    if (!p) return fail(nullptr, LBM_EINVAL, "null params");
    if (p->nx < 3 || p->ny < 3) return fail(nullptr, LBM_EINVAL, "nx and ny must be >= 3");
    if (p->nx > (1 << 28) || p->ny > (1 << 28) || (double)p->nx * (double)p->ny > 4.0e10)
        return fail(nullptr, LBM_EINVAL, "grid too large");
    if (!(p->r > 0.0) || !std::isfinite(p->r)) return fail(nullptr, LBM_EINVAL, "r must be > 0");
    if (!(p->gamma > 0.0 && p->gamma <= 1.0)) return fail(nullptr, LBM_EINVAL, "gamma must be in (0, 1]");
    if (!(p->nu > 0.0) || !std::isfinite(p->nu)) return fail(nullptr, LBM_EINVAL, "nu must be > 0");
    const double w = omega_nu_of(*p);
    if (!(w > 0.0 && w < 2.0)) return fail(nullptr, LBM_EINVAL, "omega_nu outside (0, 2)");
    if (!(p->omega_xi > 0.0 && p->omega_xi < 2.0)) return fail(nullptr, LBM_EINVAL, "omega_xi outside (0, 2)");
    if (!std::isfinite(p->u_lid) || std::fabs(p->u_lid) >= q_of(p->r) / std::sqrt(3.0))
        return fail(nullptr, LBM_EINVAL, "|u_lid| must be below the sound speed q c_s*");
    if (!std::isfinite(p->fx) || !std::isfinite(p->fy)) return fail(nullptr, LBM_EINVAL, "force not finite");
    if (!ops_for(p->dtype)) return fail(nullptr, LBM_EINVAL, "unknown dtype");
    if (p->bc < LBM_BC_CAVITY || p->bc > LBM_BC_PERIODIC) return fail(nullptr, LBM_EINVAL, "unknown bc");
    if (p->drho != LBM_DRHO_CURRENT && p->drho != LBM_DRHO_OFF) return fail(nullptr, LBM_EINVAL, "unknown drho");
    if (p->model != LBM_MODEL_PRC && p->model != LBM_MODEL_PRNR) return fail(nullptr, LBM_EINVAL, "unknown model");
    return LBM_OK;
}

lbm_status lbm_workspace_bytes(const lbm_params *p, size_t *bytes)
{
    lbm_status s = lbm_params_check(p);
    if (s != LBM_OK) return s;
    if (!bytes) return fail(nullptr, LBM_EINVAL, "null bytes");
    *bytes = make_layout(*p).total;
    return LBM_OK;
}

lbm_status lbm_omega_nu(const lbm_params *p, double *omega_nu)
{
    lbm_status s = lbm_params_check(p);
    if (s != LBM_OK) return s;
    if (!omega_nu) return fail(nullptr, LBM_EINVAL, "null out");
    *omega_nu = omega_nu_of(*p);
    return LBM_OK;
}

lbm_status lbm_create_p(const lbm_params *p, lbm_t *out)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "null out");
    *out = nullptr;
    lbm_status s = lbm_params_check(p);
    if (s != LBM_OK) return s;
    lbm_t h = new (std::nothrow) lbm_s();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    const size_t bytes = make_layout(*p).total;
    void *ws = nullptr;
    e = cudaMalloc(&ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, LBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    cudaStream_t stream;
    e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(ws);
        delete h;
        return fail(nullptr, LBM_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    s = init_handle(h, *p, ws, bytes, true, stream, true);
    if (s != LBM_OK) {
        g_err = h->err;
        lbm_destroy(h);
        return s;
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_create(int nx, int ny, double r, double gamma, double nu, double u_lid, int dtype, lbm_t *out)
{
    lbm_params p;
    lbm_params_init(&p, nx, ny, r, gamma, nu, u_lid, dtype);
    return lbm_create_p(&p, out);
}

lbm_status lbm_create_ex(const lbm_params *p, void *workspace, size_t workspace_bytes, void *stream, lbm_t *out)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "null out");
    *out = nullptr;
    lbm_status s = lbm_params_check(p);
    if (s != LBM_OK) return s;
    if (!workspace) return fail(nullptr, LBM_EINVAL, "null workspace");
    if (reinterpret_cast<uintptr_t>(workspace) % ALIGN) return fail(nullptr, LBM_EINVAL, "workspace not 256-byte aligned");
    if (workspace_bytes < make_layout(*p).total) return fail(nullptr, LBM_ENOMEM, "workspace too small");
    lbm_t h = new (std::nothrow) lbm_s();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    s = init_handle(h, *p, workspace, workspace_bytes, false, static_cast<cudaStream_t>(stream), false);
    if (s != LBM_OK) {
        g_err = h->err;
        lbm_destroy(h);
        return s;
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_set_stream(lbm_t h, void *stream)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->own_stream) CK(h, cudaStreamDestroy(h->stream));
    h->stream = static_cast<cudaStream_t>(stream);
    h->own_stream = false;
    return LBM_OK;
}

void lbm_destroy(lbm_t h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->have_g20) cudaGraphExecDestroy(h->g20);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char *lbm_last_error(lbm_t h)
{
    return h ? h->err.c_str() : g_err.c_str();
}

lbm_status lbm_step(lbm_t h, long n)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (n < 0) return fail(h, LBM_EINVAL, "negative step count");
    k_status_arm<<<1, 1, 0, h->stream>>>(h->st, -1.0);
    CK(h, cudaGetLastError());
    return enqueue_steps(h, n);
}

lbm_status lbm_run(lbm_t h, double tol, long max_steps, long *steps_done)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (max_steps < 0 || !(tol == tol)) return fail(h, LBM_EINVAL, "bad tol / max_steps");
    const long long t0 = h->t;
    long long left = max_steps;
    k_status_arm<<<1, 1, 0, h->stream>>>(h->st, tol);
    CK(h, cudaGetLastError());
    if (is_cluster(h)) {
        // one launch per chunk; the engine stops on the device at the step
        // whose residual meets tol and writes that state back
        s = read_status(h);
        if (s != LBM_OK) return s;
        long long chunk = 2000;
        while (!h->st_host->stop && left > 0) {
            const long long n = left < chunk ? left : chunk;
            s = launch_cluster(h, h->stream, h->t, n);
            if (s != LBM_OK) return s;
            s = read_status(h);
            if (s != LBM_OK) return s;
            if (h->st_host->stop && h->st_host->res_step > h->t) {
                left -= h->st_host->res_step - h->t;
                h->t = h->st_host->res_step;
            } else {
                h->t += n;
                left -= n;
            }
            if (chunk < (1LL << 20)) chunk *= 2;
        }
        if (steps_done) *steps_done = (long)(h->t - t0);
        if (h->st_host->diverged) return fail(h, LBM_EDIVERGED, "residual or mass not finite");
        if (h->st_host->converged) return LBM_OK;
        return LBM_ENOTCONVERGED;
    }
    // align to a residual boundary with single launches
    while (left > 0 && (h->t % RES_INTERVAL) != 0) {
        s = launch_one(h, h->stream, h->t);
        if (s != LBM_OK) return s;
        h->t++;
        left--;
        if ((h->t % RES_INTERVAL) == 0) {
            s = read_status(h);
            if (s != LBM_OK) return s;
            if (h->st_host->stop) break;
        }
    }
    long long batch = 8;  // graph replays per host check
    s = read_status(h);
    if (s != LBM_OK) return s;
    while (!h->st_host->stop && left >= RES_INTERVAL) {
        s = ensure_graph(h);
        if (s != LBM_OK) return s;
        long long nb = left / RES_INTERVAL;
        if (nb > batch) nb = batch;
        for (long long i = 0; i < nb; i++) CK(h, cudaGraphLaunch(h->g20, h->stream));
        s = read_status(h);
        if (s != LBM_OK) return s;
        if (h->st_host->stop) {
            const long long done = h->st_host->res_step - h->t;  // steps actually performed
            h->t = h->st_host->res_step;
            left -= done;
            break;
        }
        h->t += nb * RES_INTERVAL;
        left -= nb * RES_INTERVAL;
        if (batch < 2048) batch *= 2;
    }
    if (!h->st_host->stop && left > 0) {  // tail shorter than one residual block
        s = enqueue_steps(h, left);
        if (s != LBM_OK) return s;
        s = read_status(h);
        if (s != LBM_OK) return s;
    }
    if (steps_done) *steps_done = (long)(h->t - t0);
    if (h->st_host->diverged) return fail(h, LBM_EDIVERGED, "residual or mass not finite");
    if (h->st_host->converged) return LBM_OK;
    return LBM_ENOTCONVERGED;
}

lbm_status lbm_sync(lbm_t h)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_info(lbm_t h, lbm_info_t *info)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (!info) return fail(h, LBM_EINVAL, "null info");
    s = read_status(h);
    if (s != LBM_OK) return s;
    info->step = h->t;
    info->residual_step = h->st_host->res_step;
    info->residual = h->st_host->res_step > 0 ? h->st_host->res : INFINITY;
    info->mass = h->st_host->mass;
    info->converged = h->st_host->converged;
    info->diverged = h->st_host->diverged;
    return LBM_OK;
}

lbm_status lbm_residual(lbm_t h, double *res)
{
    if (!res) return fail(h, LBM_EINVAL, "null out");
    lbm_info_t info;
    lbm_status s = lbm_info(h, &info);
    if (s != LBM_OK) return s;
    *res = info.residual;
    return info.diverged ? LBM_EDIVERGED : LBM_OK;
}

lbm_status lbm_mass(lbm_t h, double *mass)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (!mass) return fail(h, LBM_EINVAL, "null out");
    CK(h, h->ops->mass_partial(cur_pop(h), h->gd, h->partials, h->stream));
    k_mass_final<<<1, 256, 0, h->stream>>>(h->partials, h->L.nparts, h->st, (double)h->p.nx * (double)h->p.ny);
    CK(h, cudaGetLastError());
    s = read_status(h);
    if (s != LBM_OK) return s;
    *mass = h->st_host->mass_now;
    return std::isfinite(*mass) ? LBM_OK : LBM_EDIVERGED;
}

lbm_status lbm_set_mass(lbm_t h, double mass)
{
    double now = 0.0;
    lbm_status s = lbm_mass(h, &now);
    if (s != LBM_OK) return s;
    if (!std::isfinite(mass) || !(mass > 0.0)) return fail(h, LBM_EINVAL, "mass must be finite and positive");
    const double delta = (mass - now) / ((double)h->p.nx * (double)h->p.ny);
    CK(h, h->ops->add_rest(cur_pop(h), h->gd, h->k, delta, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

// Page-locked host memory the device can address (cudaHostAlloc /
// cudaHostRegister; with unified addressing its host pointer is also its
// device pointer): kernels then read or write it directly over the host link,
// with no staging buffer and no separate copy.
bool device_addressable_host(const void *p)
{
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

lbm_status lbm_fields(lbm_t h, double *rho, double *ux, double *uy, int on_device)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    const size_t n = (size_t)h->p.nx * h->p.ny;
    if (!on_device && device_addressable_host(rho) && device_addressable_host(ux) && device_addressable_host(uy))
        on_device = 1;  // page-locked host buffers: written by the kernel itself
    if (on_device) {
        CK(h, h->ops->fields(cur_pop(h), h->gd, h->k, rho, ux, uy, nullptr, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        return LBM_OK;
    }
    DevTmp tmp;
    tmp.s = h->stream;
    CK(h, cudaMallocAsync(&tmp.p, 3 * n * sizeof(double), h->stream));
    double *d = static_cast<double *>(tmp.p);
    CK(h, h->ops->fields(cur_pop(h), h->gd, h->k, d, d + n, d + 2 * n, nullptr, h->stream));
    double *outs[3] = {rho, ux, uy};
    for (int i = 0; i < 3; i++)
        if (outs[i]) CK(h, cudaMemcpyAsync(outs[i], d + i * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_init_fields(lbm_t h, const double *rho, const double *ux, const double *uy, int on_device)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (!rho || !ux || !uy) return fail(h, LBM_EINVAL, "null field");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    DevTmp tmp;
    tmp.s = h->stream;
    const double *d[3] = {rho, ux, uy};
    if (!on_device && device_addressable_host(rho) && device_addressable_host(ux) && device_addressable_host(uy))
        on_device = 1;  // page-locked host buffers: read by the kernel itself
    if (!on_device) {
        CK(h, cudaMallocAsync(&tmp.p, 3 * n * sizeof(double), h->stream));
        double *b = static_cast<double *>(tmp.p);
        for (int i = 0; i < 3; i++) {
            CK(h, cudaMemcpyAsync(b + i * n, d[i], n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            d[i] = b + i * n;
        }
    }
    s = reset_state_meta(h);
    if (s != LBM_OK) return s;
    CK(h, h->ops->init_fields(h->pop[0], h->gd, h->k, h->p.gamma, d[0], d[1], d[2], h->snap, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_t h, const double *f, int on_device)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (!f) return fail(h, LBM_EINVAL, "null populations");
    const size_t n = 9 * (size_t)h->p.nx * h->p.ny;
    DevTmp tmp;
    tmp.s = h->stream;
    const double *d = f;
    if (!on_device) {
        CK(h, cudaMallocAsync(&tmp.p, n * sizeof(double), h->stream));
        CK(h, cudaMemcpyAsync(tmp.p, f, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        d = static_cast<const double *>(tmp.p);
    }
    s = reset_state_meta(h);
    if (s != LBM_OK) return s;
    CK(h, h->ops->set_pop(h->pop[0], h->gd, h->k, d, h->stream));
    CK(h, h->ops->fields(h->pop[0], h->gd, h->k, nullptr, nullptr, nullptr, h->snap, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_t h, double *f, int on_device)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (!f) return fail(h, LBM_EINVAL, "null populations");
    const size_t n = 9 * (size_t)h->p.nx * h->p.ny;
    if (on_device) {
        CK(h, h->ops->get_pop(cur_pop(h), h->gd, h->k, f, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        return LBM_OK;
    }
    DevTmp tmp;
    tmp.s = h->stream;
    CK(h, cudaMallocAsync(&tmp.p, n * sizeof(double), h->stream));
    CK(h, h->ops->get_pop(cur_pop(h), h->gd, h->k, static_cast<double *>(tmp.p), h->stream));
    CK(h, cudaMemcpyAsync(f, tmp.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_variant_count(int dtype, int *n)
{
    const prc::DtypeOps *ops = ops_for(dtype);
    if (!ops || !n) return fail(nullptr, LBM_EINVAL, "bad dtype / null out");
    *n = ops->nvariants;
    return LBM_OK;
}

lbm_status lbm_variant_info(int dtype, int variant, int *tile_w, int *tile_h, int *threads, int *ctas_per_sm)
{
    const prc::DtypeOps *ops = ops_for(dtype);
    if (!ops || variant < 0 || variant >= ops->nvariants) return fail(nullptr, LBM_EINVAL, "no such variant");
    const prc::Variant &v = ops->variants[variant];
    if (tile_w) *tile_w = v.w;
    if (tile_h) *tile_h = v.h;
    if (threads) *threads = v.threads;
    if (ctas_per_sm) *ctas_per_sm = v.ctas_per_sm;
    return LBM_OK;
}

lbm_status lbm_get_variant(lbm_t h, int *variant)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (!variant) return fail(h, LBM_EINVAL, "null out");
    *variant = h->variant;
    return LBM_OK;
}

lbm_status lbm_set_variant(lbm_t h, int variant)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    CK(h, cudaStreamSynchronize(h->stream));
    return apply_variant(h, variant);
}

lbm_status lbm_autotune(lbm_t h, int steps, int *best, double *ms_per_step)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (steps < 2) return fail(h, LBM_EINVAL, "autotune needs >= 2 steps");
    steps += steps & 1;  // even: the state returns to its buffer
    const int nv = h->p.model == LBM_MODEL_PRC ? h->ops->nvariants : 0;
    const int entry_variant = h->variant;
    prc::ClusterGeom cg;
    const bool cluster_ok = cluster_select(h, cg) == LBM_OK;
    h->err.clear();
    if (ms_per_step) ms_per_step[nv] = -1.0;
    CK(h, cudaStreamSynchronize(h->stream));
    // keep the state: copy the current populations, snapshot and status aside
    const long long t_keep = h->t;
    void *keep = nullptr;
    const size_t kb = h->L.pop_bytes + h->L.snap_bytes + sizeof(DevStatus);
    CK(h, cudaMallocAsync(&keep, kb, h->stream));
    char *kc = static_cast<char *>(keep);
    CK(h, cudaMemcpyAsync(kc, cur_pop(h), h->L.pop_bytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(kc + h->L.pop_bytes, h->snap, h->L.snap_bytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(kc + h->L.pop_bytes + h->L.snap_bytes, h->st, sizeof(DevStatus), cudaMemcpyDeviceToDevice,
                          h->stream));
    k_status_arm<<<1, 1, 0, h->stream>>>(h->st, -1.0);
    CK(h, cudaGetLastError());
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    int arg = entry_variant;
    double bestms = 1e300;
    lbm_status rs = LBM_OK;
    // candidates: the interior variants 0 .. nv-1, the cluster engine (when
    // the grid fits it), the general kernel
    for (int v = 0; v < nv + 2 && rs == LBM_OK; v++) {
        const int var = v < nv ? v : (v == nv ? LBM_VARIANT_CLUSTER : -1);
        if (var == LBM_VARIANT_CLUSTER && !cluster_ok) continue;
        rs = apply_variant(h, var);
        if (rs != LBM_OK) break;
        // plain steps only: a step index of 0 or 1 (same buffer parity as t)
        // never carries the residual epilogue
        const long long t0 = h->t;
        if (var == LBM_VARIANT_CLUSTER) {  // the engine runs many steps per launch
            rs = launch_cluster(h, h->stream, t0 & 1, 2);
            cudaEventRecord(e0, h->stream);
            if (rs == LBM_OK) rs = launch_cluster(h, h->stream, t0 & 1, steps);
            cudaEventRecord(e1, h->stream);
        } else {
            for (int i = 0; i < 2 && rs == LBM_OK; i++) rs = launch_one(h, h->stream, h->t & 1), h->t++;  // warm
            cudaEventRecord(e0, h->stream);
            for (int i = 0; i < steps && rs == LBM_OK; i++) rs = launch_one(h, h->stream, h->t & 1), h->t++;
            cudaEventRecord(e1, h->stream);
        }
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / steps;
        if (ms_per_step) ms_per_step[v] = per;
        if (per < bestms) {
            bestms = per;
            arg = var;
        }
        h->t = t0;  // even number of steps: the state is back in pop[t & 1]
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore the state
    h->t = t_keep;
    cudaMemcpyAsync(cur_pop(h), kc, h->L.pop_bytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(h->snap, kc + h->L.pop_bytes, h->L.snap_bytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(h->st, kc + h->L.pop_bytes + h->L.snap_bytes, sizeof(DevStatus), cudaMemcpyDeviceToDevice,
                    h->stream);
    cudaFreeAsync(keep, h->stream);
    CK(h, cudaStreamSynchronize(h->stream));
    if (rs != LBM_OK) return rs;
    if (best) *best = arg;
    return apply_variant(h, arg);
}

// ---------------------------------------------------------------------------
// Allocation-free step.  Some callers cannot call cudaMalloc: code whose
// device memory is entirely reserved by another allocator, programs that fix
// their memory budget at start-up, and latency-critical loops that cannot
// take the implicit device synchronisation of cudaMalloc / cudaFree.  lbm_step_noalloc serves
// them: the only scratch it needs (per-CTA FP64 partial sums and a status
// word) lives in the file-scope device arrays below, which every GPU that
// loads this library holds until the process exits.

namespace {

constexpr int NOALLOC_MAX_PARTS = 16384;  // 256 KiB of double2: ceil(nx/32) * ceil(ny/8) CTAs at most
static __device__ __align__(256) double2 g_noalloc_partials[NOALLOC_MAX_PARTS];
static __device__ __align__(256) DevStatus g_noalloc_status;

struct NoallocScratch {
    double2 *partials;
    DevStatus *status;
};

std::mutex g_noalloc_mu;
std::map<int, NoallocScratch> g_noalloc_addr;  // device ordinal -> device addresses of the arrays

// Device addresses of the scratch arrays on the current device.  In host code
// the array names are host-side stand-ins, not device addresses; the real
// addresses come from cudaGetSymbolAddress with the device current, once per
// device.  They stay valid for the life of the device's primary context; a
// device reset ends that context, and the entry point's contract excludes
// calls after one.
lbm_status noalloc_scratch(NoallocScratch *out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) {
        *out = it->second;
        return LBM_OK;
    }
    NoallocScratch sc;
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&sc.partials), g_noalloc_partials);
    if (e != cudaSuccess)
        return fail(nullptr, LBM_ECUDA, std::string("cudaGetSymbolAddress(partials): ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&sc.status), g_noalloc_status);
    if (e != cudaSuccess)
        return fail(nullptr, LBM_ECUDA, std::string("cudaGetSymbolAddress(status): ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = sc;
    *out = sc;
    return LBM_OK;
}

__global__ void __launch_bounds__(256) k_noalloc_finalize(const double2 *partials, int n, double *out, double nnodes)
{
    double a, b;
    reduce_partials(partials, n, a, b);
    if (threadIdx.x == 0) {
        out[0] = sqrt(a);
        out[1] = nnodes + b;
    }
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_params *p, const void *src, void *dst, void *snap, int with_residual,
                                       double *out, void *stream)
{
    lbm_status s = lbm_params_check(p);
    if (s != LBM_OK) return s;
    if (!src || !dst || !snap) return fail(nullptr, LBM_EINVAL, "null buffer");
    if (with_residual && !out) return fail(nullptr, LBM_EINVAL, "null residual output");
    if (src == dst) return fail(nullptr, LBM_EINVAL, "src and dst must be different buffers");
    const Plan pl = make_plan(*p, 0, -1);  // general kernel over the whole grid
    const long long cells = (long long)((p->nx + 31) / 32) * (long long)((p->ny + 7) / 8);
    if (cells > NOALLOC_MAX_PARTS || pl.nparts > NOALLOC_MAX_PARTS)
        return fail(nullptr, LBM_EINVAL,
                    "grid too large for lbm_step_noalloc: ceil(nx/32)*ceil(ny/8) = " + std::to_string(cells) +
                        " exceeds " + std::to_string(NOALLOC_MAX_PARTS));
    NoallocScratch sc;
    s = noalloc_scratch(&sc);
    if (s != LBM_OK) return s;
    const prc::DtypeOps *ops = ops_for(p->dtype);
    const Layout L = make_layout(*p);
    const Grid gd = make_grid(*p, L);
    Coef<double> k;
    make_coef(*p, k);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the status word shared by every call must start clear (stop = 0)
    cudaError_t e = cudaMemsetAsync(sc.status, 0, sizeof(DevStatus), st);
    if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    e = ops->step_general(src, dst, pl, gd, k, snap, sc.partials, sc.status, p->drho == LBM_DRHO_CURRENT,
                          with_residual != 0, p->fx != 0.0 || p->fy != 0.0, st);
    if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, std::string("step launch: ") + cudaGetErrorString(e));
    if (with_residual) {
        k_noalloc_finalize<<<1, 256, 0, st>>>(sc.partials, pl.nparts, out, (double)p->nx * (double)p->ny);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, std::string("finalize launch: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}

namespace {
struct SaveHeader {
    char magic[8];
    int32_t version, nx, ny, dtype;
    int64_t t;
    DevStatus st;
    uint64_t pop_bytes, snap_bytes;
};
}  // namespace

lbm_status lbm_save_bytes(lbm_t h, size_t *bytes)
{
    lbm_status s = enter(h);
    if (s != LBM_OK) return s;
    if (!bytes) return fail(h, LBM_EINVAL, "null out");
    *bytes = sizeof(SaveHeader) + h->L.pop_bytes + h->L.snap_bytes;
    return LBM_OK;
}

lbm_status lbm_save(lbm_t h, void *host_buf, size_t n)
{
    size_t need = 0;
    lbm_status s = lbm_save_bytes(h, &need);
    if (s != LBM_OK) return s;
    if (!host_buf || n < need) return fail(h, LBM_EINVAL, "checkpoint buffer too small");
    s = read_status(h);
    if (s != LBM_OK) return s;
    SaveHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "PRCLBM1", 8);
    hd.version = 1;
    hd.nx = h->p.nx;
    hd.ny = h->p.ny;
    hd.dtype = h->p.dtype;
    hd.t = h->t;
    hd.st = *h->st_host;
    hd.pop_bytes = h->L.pop_bytes;
    hd.snap_bytes = h->L.snap_bytes;
    char *b = static_cast<char *>(host_buf);
    std::memcpy(b, &hd, sizeof(hd));
    CK(h, cudaMemcpyAsync(b + sizeof(hd), cur_pop(h), h->L.pop_bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(b + sizeof(hd) + h->L.pop_bytes, h->snap, h->L.snap_bytes, cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_load(lbm_t h, const void *host_buf, size_t n)
{
    size_t need = 0;
    lbm_status s = lbm_save_bytes(h, &need);
    if (s != LBM_OK) return s;
    if (!host_buf || n < need) return fail(h, LBM_EINVAL, "checkpoint buffer too small");
    SaveHeader hd;
    std::memcpy(&hd, host_buf, sizeof(hd));
    if (std::memcmp(hd.magic, "PRCLBM1", 8) != 0 || hd.version != 1 || hd.nx != h->p.nx || hd.ny != h->p.ny ||
        hd.dtype != h->p.dtype || hd.pop_bytes != h->L.pop_bytes || hd.snap_bytes != h->L.snap_bytes)
        return fail(h, LBM_EINVAL, "checkpoint does not match this handle");
    const char *b = static_cast<const char *>(host_buf);
    CK(h, cudaStreamSynchronize(h->stream));
    h->t = hd.t;
    CK(h, cudaMemcpyAsync(cur_pop(h), b + sizeof(hd), h->L.pop_bytes, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->snap, b + sizeof(hd) + h->L.pop_bytes, h->L.snap_bytes, cudaMemcpyHostToDevice,
                          h->stream));
    *h->st_host = hd.st;
    CK(h, cudaMemcpyAsync(h->st, h->st_host, sizeof(DevStatus), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

}  // extern "C"
