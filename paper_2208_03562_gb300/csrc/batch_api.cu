// batch_api.cu -- C ABI of the batched engine (include/prc_lbm.h, lbm_batch_*).
//
// A batch holds up to `capacity` independent instances (slots).  Each slot
// owns its device memory (two population sets and a residual snapshot,
// allocated stream-ordered when the slot is filled and released when it is
// removed), its parameters, tolerance and step limit.  lbm_batch_launch
// advances every active slot with one persistent cooperative launch of
// k_batch (optionally through a captured CUDA graph); slots retire on the
// device as they converge, diverge or reach their step limit.  Slots can be
// added and removed between launches, which is what continuous batching
// needs.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "prc_host.h"
#include "prc_lbm.h"
#include "prc_ops.h"

using namespace prc_host;
using prc::BatchCtl;
using prc::BatchDyn;
using prc::BatchInst;

namespace {

struct Slot {
    bool used = false;
    lbm_params p;
    Layout L;
    Grid gd;
    Coef<double> k;
    void *mem = nullptr;
    double tol = 0.0;
    long long max_steps = 0;
    long long stall_window = 0;
    double stall_ratio = 0.0;
};

thread_local std::string g_batch_err;

}  // namespace

struct lbm_batch_s {
    int dtype;
    const prc::DtypeOps *ops;
    int capacity;
    int device;
    int num_sms;
    int occupancy;
    cudaStream_t stream;
    bool own_stream;
    std::vector<Slot> slots;
    char *d_tables;       // coefficients, dynamic state, control word, instance list
    void *d_coefs;
    BatchDyn *d_dyn;
    BatchCtl *d_ctl;
    BatchInst *d_inst;
    BatchDyn *h_dyn;      // pinned mirrors
    BatchInst *h_inst;
    BatchCtl *h_ctl;
    char *h_coef;         // staging for one slot's coefficients (pinned)
    double2 *d_partials;
    size_t part_cap;
    bool in_flight;
    cudaGraphExec_t gexec;
    bool have_gexec;
    long long next_limit;  // lbm_batch_set_wait_limit, for the next launch only
    int next_hold;
    int ctas_per_sm;       // persistent grid: ctas_per_sm x SMs (0: occupancy)
    // TMA-staged body (k_batch_tma)
    CUtensorMap *d_tmaps;  // four load descriptors per slot: interior box of pop[0], pop[1]; wall box of both
    CUtensorMap *h_tmaps;  // pinned staging of one slot's four
    int occupancy_tma;     // resident CTAs per SM of k_batch_tma (0: not available)
    int body;              // LBM_BATCH_BODY_*
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch_t b, lbm_status s, const std::string &msg)
{
    if (b) b->err = msg;
    else g_batch_err = msg;
    return s;
}

#define BCK(b, call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return bfail(b, LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

lbm_status benter(lbm_batch_t b)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "null batch");
    b->err.clear();
    BCK(b, cudaSetDevice(b->device));
    return LBM_OK;
}

size_t slot_bytes(const Layout &L) { return 2 * L.pop_bytes + L.snap_bytes; }

void *slot_pop(const Slot &s, int i) { return static_cast<char *>(s.mem) + i * s.L.pop_bytes; }
void *slot_snap(const Slot &s) { return static_cast<char *>(s.mem) + 2 * s.L.pop_bytes; }

lbm_status check_slot(lbm_batch_t b, int slot)
{
    if (slot < 0 || slot >= b->capacity || !b->slots[slot].used) return bfail(b, LBM_EINVAL, "no such slot");
    if (b->in_flight) return bfail(b, LBM_EINVAL, "a launch is in flight: call lbm_batch_wait first");
    return LBM_OK;
}

// Every active slot allows the specialised body (density-gradient terms, no
// force, central moments)?
bool all_spec(lbm_batch_t b)
{
    bool any = false;
    for (int i = 0; i < b->capacity; i++) {
        const Slot &sl = b->slots[i];
        if (!sl.used || b->h_dyn[i].state != prc::BATCH_ACTIVE) continue;
        any = true;
        if (sl.p.drho != LBM_DRHO_CURRENT || sl.p.fx != 0.0 || sl.p.fy != 0.0 || sl.p.model != LBM_MODEL_PRC ||
            sl.p.bc != LBM_BC_CAVITY)
            return false;
    }
    return any;
}

// The next launch runs the TMA-staged body: allowed by the body setting, built
// for this storage type, and every active slot takes the specialised body.
bool next_is_tma(lbm_batch_t b)
{
    if (b->body == LBM_BATCH_BODY_GENERAL || b->occupancy_tma <= 0 || !all_spec(b)) return false;
    int n = 0;  // the TMA-staged body keeps a table of the launch's instances in shared memory
    for (int i = 0; i < b->capacity; i++)
        if (b->slots[i].used && b->h_dyn[i].state == prc::BATCH_ACTIVE) n++;
    return n <= prc::BT_MAX_INST;
}

int max_ctas(lbm_batch_t b) { return next_is_tma(b) ? b->occupancy_tma : b->occupancy; }

}  // namespace

extern "C" {

lbm_status lbm_batch_instance_bytes(const lbm_params *p, size_t *bytes)
{
    lbm_status s = lbm_params_check(p);
    if (s != LBM_OK) return s;
    if (!bytes) return bfail(nullptr, LBM_EINVAL, "null out");
    *bytes = slot_bytes(make_layout(*p));
    return LBM_OK;
}

lbm_status lbm_batch_create(int capacity, int dtype, void *stream, lbm_batch_t *out)
{
    if (!out) return bfail(nullptr, LBM_EINVAL, "null out");
    *out = nullptr;
    const prc::DtypeOps *ops = ops_for(dtype);
    if (!ops) return bfail(nullptr, LBM_EINVAL, "unknown dtype");
    if (capacity < 1 || capacity > 65536) return bfail(nullptr, LBM_EINVAL, "capacity must be in [1, 65536]");
    lbm_batch_t b = new (std::nothrow) lbm_batch_s();
    if (!b) return bfail(nullptr, LBM_ENOMEM, "host allocation failed");
    b->dtype = dtype;
    b->ops = ops;
    b->capacity = capacity;
    b->slots.resize(capacity);
    auto bail = [&](lbm_status s) {
        g_batch_err = b->err;
        lbm_batch_destroy(b);
        return s;
    };
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) {
        b->err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return bail(LBM_ECUDA);
    }
    if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
        ops->batch_occupancy(&b->occupancy) != cudaSuccess || b->occupancy < 1) {
        b->err = "occupancy query failed";
        return bail(LBM_ECUDA);
    }
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            b->err = "stream creation failed";
            return bail(LBM_ECUDA);
        }
        b->own_stream = true;
    }
    if (ops->batch_tma_prepare) {  // the TMA-staged body: shared-memory opt-in, occupancy
        if (ops->batch_tma_prepare() != cudaSuccess || ops->batch_tma_occupancy(&b->occupancy_tma) != cudaSuccess) {
            cudaGetLastError();
            b->occupancy_tma = 0;
        }
    }
    const size_t cbytes = align_up((size_t)capacity * ops->coef_bytes, ALIGN);
    const size_t dbytes = align_up((size_t)capacity * sizeof(BatchDyn), ALIGN);
    const size_t ibytes = align_up((size_t)capacity * sizeof(BatchInst), ALIGN);
    const size_t mbytes = b->occupancy_tma > 0 ? align_up((size_t)capacity * 4 * sizeof(CUtensorMap), ALIGN) : 0;
    const size_t tbytes = cbytes + dbytes + ALIGN + ibytes + mbytes;
    if (cudaMalloc(&b->d_tables, tbytes) != cudaSuccess) {
        cudaGetLastError();
        b->err = "device allocation of the batch tables failed";
        return bail(LBM_ENOMEM);
    }
    b->d_coefs = b->d_tables;
    b->d_dyn = reinterpret_cast<BatchDyn *>(b->d_tables + cbytes);
    b->d_ctl = reinterpret_cast<BatchCtl *>(b->d_tables + cbytes + dbytes);
    b->d_inst = reinterpret_cast<BatchInst *>(b->d_tables + cbytes + dbytes + ALIGN);
    b->d_tmaps = mbytes ? reinterpret_cast<CUtensorMap *>(b->d_tables + cbytes + dbytes + ALIGN + ibytes) : nullptr;
    if ((mbytes && cudaMallocHost(&b->h_tmaps, 4 * sizeof(CUtensorMap)) != cudaSuccess) ||
        cudaMallocHost(&b->h_dyn, capacity * sizeof(BatchDyn)) != cudaSuccess ||
        cudaMallocHost(&b->h_inst, capacity * sizeof(BatchInst)) != cudaSuccess ||
        cudaMallocHost(&b->h_ctl, sizeof(BatchCtl)) != cudaSuccess ||
        cudaMallocHost(&b->h_coef, ops->coef_bytes) != cudaSuccess) {
        b->err = "pinned host allocation failed";
        return bail(LBM_ENOMEM);
    }
    for (int i = 0; i < capacity; i++) {
        std::memset(&b->h_dyn[i], 0, sizeof(BatchDyn));
        b->h_dyn[i].state = prc::BATCH_EMPTY;
    }
    if (cudaMemcpyAsync(b->d_dyn, b->h_dyn, capacity * sizeof(BatchDyn), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        b->err = "table initialisation failed";
        return bail(LBM_ECUDA);
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch_t b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->have_gexec) cudaGraphExecDestroy(b->gexec);
    for (auto &s : b->slots)
        if (s.mem) cudaFreeAsync(s.mem, b->stream);
    if (b->d_partials) cudaFreeAsync(b->d_partials, b->stream);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->d_tables) cudaFree(b->d_tables);
    if (b->h_dyn) cudaFreeHost(b->h_dyn);
    if (b->h_inst) cudaFreeHost(b->h_inst);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->h_coef) cudaFreeHost(b->h_coef);
    if (b->h_tmaps) cudaFreeHost(b->h_tmaps);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *lbm_batch_last_error(lbm_batch_t b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

lbm_status lbm_batch_add(lbm_batch_t b, const lbm_params *p, double tol, long max_steps, int *slot)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    s = lbm_params_check(p);
    if (s != LBM_OK) return bfail(b, s, lbm_last_error(nullptr));
    if (p->dtype != b->dtype) return bfail(b, LBM_EINVAL, "instance dtype differs from the batch dtype");
    if (max_steps < 1 || !(tol == tol)) return bfail(b, LBM_EINVAL, "bad tol / max_steps");
    if (b->in_flight) return bfail(b, LBM_EINVAL, "a launch is in flight: call lbm_batch_wait first");
    int k = -1;
    for (int i = 0; i < b->capacity; i++)
        if (!b->slots[i].used) {
            k = i;
            break;
        }
    if (k < 0) return bfail(b, LBM_ENOMEM, "no free slot");
    Slot &sl = b->slots[k];
    sl.p = *p;
    sl.L = make_layout(*p);
    sl.gd = make_grid(*p, sl.L);
    make_coef(*p, sl.k);
    sl.tol = tol;
    sl.max_steps = max_steps;
    sl.stall_window = 0;
    sl.stall_ratio = 0.0;
    cudaError_t e = cudaMallocAsync(&sl.mem, slot_bytes(sl.L), b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sl.mem = nullptr;
        return bfail(b, LBM_ENOMEM, std::string("instance allocation failed: ") + cudaGetErrorString(e));
    }
    // rest state (shifted storage 0) and the snapshot of its u_x
    BCK(b, cudaMemsetAsync(sl.mem, 0, slot_bytes(sl.L), b->stream));
    BCK(b, b->ops->fields(slot_pop(sl, 0), sl.gd, sl.k, nullptr, nullptr, nullptr, slot_snap(sl), b->stream));
    if (b->d_tmaps) {  // load descriptors of the slot's two sets for the TMA body: interior and wall boxes
        for (int q = 0; q < 4; q++) {
            const CUresult r = encode_pop_map(&b->h_tmaps[q], b->ops->elem, slot_pop(sl, q & 1), sl.p.nx, sl.p.ny,
                                              sl.L.pitch, sl.L.plane, prc::BT_W + 2 * b->ops->tma_padx,
                                              q < 2 ? prc::BT_H + 2 : prc::BT_H + 4, CU_TENSOR_MAP_L2_PROMOTION_L2_256B);
            if (r != CUDA_SUCCESS) {
                cudaFreeAsync(sl.mem, b->stream);
                sl.mem = nullptr;
                return bfail(b, LBM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
            }
        }
        BCK(b, cudaMemcpyAsync(b->d_tmaps + 4 * k, b->h_tmaps, 4 * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                               b->stream));
    }
    b->ops->coef_convert(sl.k, b->h_coef);
    BCK(b, cudaMemcpyAsync(static_cast<char *>(b->d_coefs) + (size_t)k * b->ops->coef_bytes, b->h_coef,
                           b->ops->coef_bytes, cudaMemcpyHostToDevice, b->stream));
    BatchDyn &d = b->h_dyn[k];
    std::memset(&d, 0, sizeof(d));
    d.res = INFINITY;
    d.state = prc::BATCH_ACTIVE;
    BCK(b, cudaMemcpyAsync(b->d_dyn + k, &d, sizeof(BatchDyn), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));  // the pinned staging buffers are reused
    sl.used = true;
    if (slot) *slot = k;
    return LBM_OK;
}

lbm_status lbm_batch_set_stall(lbm_batch_t b, int slot, long window, double ratio)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    s = check_slot(b, slot);
    if (s != LBM_OK) return s;
    if (window < 0 || (window > 0 && !(ratio > 0.0))) return bfail(b, LBM_EINVAL, "bad stall window / ratio");
    Slot &sl = b->slots[slot];
    sl.stall_window = window;
    sl.stall_ratio = window > 0 ? ratio : 0.0;
    return LBM_OK;
}

lbm_status lbm_batch_set_wait_limit(lbm_batch_t b, long long cycles, int hold)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    if (cycles < 0) return bfail(b, LBM_EINVAL, "wait limit must be >= 0");
    b->next_limit = cycles;
    b->next_hold = hold != 0;
    return LBM_OK;
}

lbm_status lbm_batch_remove(lbm_batch_t b, int slot)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    s = check_slot(b, slot);
    if (s != LBM_OK) return s;
    Slot &sl = b->slots[slot];
    BCK(b, cudaFreeAsync(sl.mem, b->stream));
    sl.mem = nullptr;
    sl.used = false;
    b->h_dyn[slot].state = prc::BATCH_EMPTY;
    BCK(b, cudaMemcpyAsync(b->d_dyn + slot, &b->h_dyn[slot], sizeof(BatchDyn), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

lbm_status lbm_batch_launch(lbm_batch_t b, long steps, int use_graph)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    if (b->in_flight) return bfail(b, LBM_EINVAL, "a launch is in flight: call lbm_batch_wait first");
    if (steps < 1 || steps > (1L << 30)) return bfail(b, LBM_EINVAL, "steps must be in [1, 2^30]");
    const bool tma = next_is_tma(b);
    // compact list of the active slots, tiles in slot order
    int n = 0, tiles = 0;
    for (int i = 0; i < b->capacity; i++) {
        const Slot &sl = b->slots[i];
        if (!sl.used || b->h_dyn[i].state != prc::BATCH_ACTIVE) continue;
        BatchInst &I = b->h_inst[n++];
        std::memset(&I, 0, sizeof(I));
        I.slot = i;
        I.pop[0] = slot_pop(sl, 0);
        I.pop[1] = slot_pop(sl, 1);
        I.snap = slot_snap(sl);
        I.gd = sl.gd;
        // the tile shape of k_batch: 64 x 8 (pairs, FP32 collision) or 32 x 8 (FP64)
        I.tiles_x = ceil_div(sl.p.nx, sl.p.dtype == LBM_F64 ? prc::BX : prc::PTW);
        I.tiles = I.tiles_x * ceil_div(sl.p.ny, prc::BY);
        I.tile_start = tiles;
        I.part_base = tiles;
        I.t0 = b->h_dyn[i].t;
        I.drho = sl.p.drho == LBM_DRHO_CURRENT;
        I.force = sl.p.fx != 0.0 || sl.p.fy != 0.0;
        I.tol = sl.tol;
        I.max_steps = sl.max_steps;
        I.stall_window = sl.stall_window;
        I.stall_ratio = sl.stall_ratio;
        if (tma) I.tmap = b->d_tmaps + 4 * i;  // the same 64 x 8 tiles, staged through the slot's descriptors
        tiles += I.tiles;
    }
    if (n == 0) return LBM_OK;  // nothing to do
    int spec = 1;  // every active slot: density-gradient terms, no force, central moments
    for (int q = 0; q < n; q++) {
        const BatchInst &I = b->h_inst[q];
        if (!I.drho || I.force || I.gd.model != LBM_MODEL_PRC) spec = 0;
    }
    if ((size_t)tiles > b->part_cap) {
        if (b->d_partials) BCK(b, cudaFreeAsync(b->d_partials, b->stream));
        b->d_partials = nullptr;
        size_t cap = (size_t)tiles + (size_t)tiles / 4;
        cudaError_t e = cudaMallocAsync(&b->d_partials, cap * sizeof(double2), b->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->part_cap = 0;
            return bfail(b, LBM_ENOMEM, "partial-sum allocation failed");
        }
        b->part_cap = cap;
    }
    BCK(b, cudaMemcpyAsync(b->d_inst, b->h_inst, n * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemsetAsync(b->d_ctl, 0, sizeof(BatchCtl), b->stream));
    if (b->next_limit > 0 || b->next_hold) {  // one launch only (lbm_batch_set_wait_limit)
        std::memset(b->h_ctl, 0, sizeof(BatchCtl));
        b->h_ctl->limit = b->next_limit;
        b->h_ctl->hold = b->next_hold;
        BCK(b, cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, b->stream));
        b->next_limit = 0;
        b->next_hold = 0;
    }
    const int occ = tma ? b->occupancy_tma : b->occupancy;
    int grid = (b->ctas_per_sm > 0 && b->ctas_per_sm < occ ? b->ctas_per_sm : occ) * b->num_sms;
    if (grid > tiles) grid = tiles;
    const int st = (int)steps;
    auto do_launch = [&](cudaStream_t ls) -> cudaError_t {
        if (tma)
            return b->ops->batch_tma_launch(b->d_inst, b->d_coefs, b->d_dyn, n, tiles, b->d_partials,
                                            b->d_ctl, st, grid, ls);
        return b->ops->batch_launch(b->d_inst, b->d_coefs, b->d_dyn, n, tiles, b->d_partials, b->d_ctl, st, grid,
                                    spec, ls);
    };
    if (use_graph) {
        cudaStream_t cs;
        BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = do_launch(cs);
            e = cudaStreamEndCapture(cs, &g);
            if (el != cudaSuccess) e = el;
        }
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(b, LBM_ECUDA, std::string("graph capture of the batch launch: ") + cudaGetErrorString(e));
        }
        if (b->have_gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->have_gexec = false;
        }
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        b->have_gexec = true;
        BCK(b, cudaGraphLaunch(b->gexec, b->stream));
    } else {
        BCK(b, do_launch(b->stream));
    }
    b->in_flight = true;
    return LBM_OK;
}

lbm_status lbm_batch_set_ctas_per_sm(lbm_batch_t b, int ctas_per_sm)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    const int occ = b->occupancy > b->occupancy_tma ? b->occupancy : b->occupancy_tma;
    if (ctas_per_sm < 0 || ctas_per_sm > occ)
        return bfail(b, LBM_EINVAL, "ctas_per_sm must be in [0, " + std::to_string(occ) + "]");
    b->ctas_per_sm = ctas_per_sm;
    return LBM_OK;
}

lbm_status lbm_batch_set_body(lbm_batch_t b, int body)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    if (body != LBM_BATCH_BODY_AUTO && body != LBM_BATCH_BODY_GENERAL)
        return bfail(b, LBM_EINVAL, "body must be LBM_BATCH_BODY_AUTO or LBM_BATCH_BODY_GENERAL");
    b->body = body;
    return LBM_OK;
}

lbm_status lbm_batch_get_body(lbm_batch_t b, int *tma)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    if (!tma) return bfail(b, LBM_EINVAL, "null out");
    *tma = next_is_tma(b) ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_batch_get_ctas_per_sm(lbm_batch_t b, int *ctas_per_sm, int *max_ctas_per_sm)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "null batch");
    const int occ = max_ctas(b);
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm > 0 && b->ctas_per_sm < occ ? b->ctas_per_sm : occ;
    if (max_ctas_per_sm) *max_ctas_per_sm = occ;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch_t b, int steps, int *best, double *ms_per_step)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    if (b->in_flight) return bfail(b, LBM_EINVAL, "a launch is in flight: call lbm_batch_wait first");
    if (steps < 1 || steps > 100000) return bfail(b, LBM_EINVAL, "steps must be in [1, 100000]");
    const int occ = max_ctas(b);
    const int current = b->ctas_per_sm > 0 && b->ctas_per_sm < occ ? b->ctas_per_sm : occ;
    // the state a launch changes: the active slots' memory and the dynamic table
    std::vector<int> act;
    size_t bytes = 0;
    for (int i = 0; i < b->capacity; i++)
        if (b->slots[i].used && b->h_dyn[i].state == prc::BATCH_ACTIVE) {
            act.push_back(i);
            bytes += slot_bytes(b->slots[i].L);
        }
    if (act.empty()) {
        if (best) *best = current;
        return LBM_OK;
    }
    const size_t dyn_bytes = (size_t)b->capacity * sizeof(BatchDyn);
    char *save = nullptr;
    if (cudaMallocAsync(&save, bytes + dyn_bytes, b->stream) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, LBM_ENOMEM, "device allocation of the state copy failed");
    }
    const std::vector<BatchDyn> h_save(b->h_dyn, b->h_dyn + b->capacity);
    auto copy_state = [&](bool out) -> cudaError_t {
        size_t off = 0;
        for (int i : act) {
            const size_t n = slot_bytes(b->slots[i].L);
            void *dev = b->slots[i].mem;
            cudaError_t e = out ? cudaMemcpyAsync(save + off, dev, n, cudaMemcpyDeviceToDevice, b->stream)
                                : cudaMemcpyAsync(dev, save + off, n, cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) return e;
            off += n;
        }
        if (!out) std::memcpy(b->h_dyn, h_save.data(), dyn_bytes);
        return out ? cudaMemcpyAsync(save + bytes, b->d_dyn, dyn_bytes, cudaMemcpyDeviceToDevice, b->stream)
                   : cudaMemcpyAsync(b->d_dyn, save + bytes, dyn_bytes, cudaMemcpyDeviceToDevice, b->stream);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lbm_status rs = LBM_OK;
    std::string msg;
    int best_c = current;
    double best_ms = 0.0;
    if (copy_state(true) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rs = LBM_ECUDA;
        msg = "set-up of the timing failed";
    }
    for (int c = 1; rs == LBM_OK && c <= occ; c++) {
        b->ctas_per_sm = c;
        float ms = 0.f;
        // one untimed launch, then a timed one, each from the saved state
        for (int rep = 0; rep < 2 && rs == LBM_OK; rep++) {
            if (copy_state(false) != cudaSuccess) {
                rs = LBM_ECUDA;
                msg = "restore of the state failed";
                break;
            }
            if (rep == 1 && cudaEventRecord(e0, b->stream) != cudaSuccess) rs = LBM_ECUDA;
            if (rs == LBM_OK) rs = lbm_batch_launch(b, steps, 0);
            if (rs == LBM_OK && rep == 1 && cudaEventRecord(e1, b->stream) != cudaSuccess) rs = LBM_ECUDA;
            if (rs == LBM_OK) rs = lbm_batch_wait(b, nullptr);
            if (rs != LBM_OK) msg = b->err.empty() ? "timing launch failed" : b->err;
        }
        if (rs == LBM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rs = LBM_ECUDA;
            msg = "event timing failed";
        }
        if (rs != LBM_OK) break;
        const double per = (double)ms / steps;
        if (ms_per_step) ms_per_step[c - 1] = per;
        if (c == 1 || per < best_ms) {
            best_ms = per;
            best_c = c;
        }
    }
    b->in_flight = false;
    const cudaError_t er = copy_state(false);
    const cudaError_t es = cudaStreamSynchronize(b->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(save, b->stream);
    cudaStreamSynchronize(b->stream);
    if (rs == LBM_OK && (er != cudaSuccess || es != cudaSuccess)) {
        rs = LBM_ECUDA;
        msg = "restore of the state failed";
    }
    b->ctas_per_sm = rs == LBM_OK ? best_c : (current == occ ? 0 : current);
    if (rs != LBM_OK) return bfail(b, rs, "lbm_batch_autotune: " + msg);
    if (best) *best = best_c;
    return LBM_OK;
}

lbm_status lbm_batch_wait(lbm_batch_t b, int *n_active)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    BCK(b, cudaMemcpyAsync(b->h_dyn, b->d_dyn, b->capacity * sizeof(BatchDyn), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    b->in_flight = false;
    int act = 0;
    for (int i = 0; i < b->capacity; i++)
        if (b->slots[i].used && b->h_dyn[i].state == prc::BATCH_ACTIVE) act++;
    if (n_active) *n_active = act;
    if (b->h_ctl->error) return bfail(b, LBM_ETIMEOUT, "grid barrier of the batch launch timed out");
    return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch_t b, long steps, int *n_active)
{
    lbm_status s = lbm_batch_launch(b, steps, 1);
    if (s != LBM_OK) return s;
    return lbm_batch_wait(b, n_active);
}

lbm_status lbm_batch_query(lbm_batch_t b, int slot, lbm_info_t *info, int *state)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    s = check_slot(b, slot);
    if (s != LBM_OK) return s;
    const BatchDyn &d = b->h_dyn[slot];
    if (info) {
        info->step = d.t;
        info->residual_step = d.res_step;
        info->residual = d.res_step > 0 ? d.res : INFINITY;
        info->mass = d.mass;
        info->converged = d.state == prc::BATCH_CONVERGED;
        info->diverged = d.state == prc::BATCH_DIVERGED;
    }
    if (state) *state = d.state;
    return LBM_OK;
}

lbm_status lbm_batch_fields(lbm_batch_t b, int slot, double *rho, double *ux, double *uy, int on_device)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    s = check_slot(b, slot);
    if (s != LBM_OK) return s;
    const Slot &sl = b->slots[slot];
    void *cur = slot_pop(sl, (int)(b->h_dyn[slot].t & 1));
    const size_t n = (size_t)sl.p.nx * sl.p.ny;
    if (on_device) {
        BCK(b, b->ops->fields(cur, sl.gd, sl.k, rho, ux, uy, nullptr, b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        return LBM_OK;
    }
    void *tmp = nullptr;
    BCK(b, cudaMallocAsync(&tmp, 3 * n * sizeof(double), b->stream));
    double *d = static_cast<double *>(tmp);
    cudaError_t e = b->ops->fields(cur, sl.gd, sl.k, d, d + n, d + 2 * n, nullptr, b->stream);
    double *outs[3] = {rho, ux, uy};
    for (int i = 0; i < 3 && e == cudaSuccess; i++)
        if (outs[i]) e = cudaMemcpyAsync(outs[i], d + i * n, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    cudaFreeAsync(tmp, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("fields: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_batch_set_populations(lbm_batch_t b, int slot, const double *f, int on_device)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    s = check_slot(b, slot);
    if (s != LBM_OK) return s;
    if (!f) return bfail(b, LBM_EINVAL, "null populations");
    Slot &sl = b->slots[slot];
    const size_t n = 9 * (size_t)sl.p.nx * sl.p.ny;
    void *tmp = nullptr;
    const double *d = f;
    if (!on_device) {
        BCK(b, cudaMallocAsync(&tmp, n * sizeof(double), b->stream));
        BCK(b, cudaMemcpyAsync(tmp, f, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
        d = static_cast<const double *>(tmp);
    }
    BCK(b, b->ops->set_pop(slot_pop(sl, 0), sl.gd, sl.k, d, b->stream));
    BCK(b, b->ops->fields(slot_pop(sl, 0), sl.gd, sl.k, nullptr, nullptr, nullptr, slot_snap(sl), b->stream));
    if (tmp) BCK(b, cudaFreeAsync(tmp, b->stream));
    BatchDyn &dd = b->h_dyn[slot];
    std::memset(&dd, 0, sizeof(dd));
    dd.res = INFINITY;
    dd.state = prc::BATCH_ACTIVE;
    BCK(b, cudaMemcpyAsync(b->d_dyn + slot, &dd, sizeof(BatchDyn), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

lbm_status lbm_batch_mass(lbm_batch_t b, int slot, double *mass)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    s = check_slot(b, slot);
    if (s != LBM_OK) return s;
    if (!mass) return bfail(b, LBM_EINVAL, "null out");
    const Slot &sl = b->slots[slot];
    const dim3 g = prc::step_grid(sl.gd);
    const size_t np = (size_t)g.x * g.y;
    void *tmp = nullptr;
    BCK(b, cudaMallocAsync(&tmp, np * sizeof(double2), b->stream));
    std::vector<double2> h(np);
    cudaError_t e = b->ops->mass_partial(slot_pop(sl, (int)(b->h_dyn[slot].t & 1)), sl.gd,
                                         static_cast<double2 *>(tmp), b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), tmp, np * sizeof(double2), cudaMemcpyDeviceToHost, b->stream);
    cudaFreeAsync(tmp, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("mass: ") + cudaGetErrorString(e));
    double m = 0.0;
    for (size_t i = 0; i < np; i++) m += h[i].y;  // fixed order
    *mass = (double)sl.p.nx * (double)sl.p.ny + m;
    return std::isfinite(*mass) ? LBM_OK : LBM_EDIVERGED;
}

lbm_status lbm_batch_set_mass(lbm_batch_t b, int slot, double mass)
{
    double now = 0.0;
    lbm_status s = lbm_batch_mass(b, slot, &now);
    if (s != LBM_OK) return s;
    if (!std::isfinite(mass) || !(mass > 0.0)) return bfail(b, LBM_EINVAL, "mass must be finite and positive");
    const Slot &sl = b->slots[slot];
    const double delta = (mass - now) / ((double)sl.p.nx * (double)sl.p.ny);
    BCK(b, b->ops->add_rest(slot_pop(sl, (int)(b->h_dyn[slot].t & 1)), sl.gd, sl.k, delta, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

lbm_status lbm_batch_get_populations(lbm_batch_t b, int slot, double *f, int on_device)
{
    lbm_status s = benter(b);
    if (s != LBM_OK) return s;
    s = check_slot(b, slot);
    if (s != LBM_OK) return s;
    if (!f) return bfail(b, LBM_EINVAL, "null populations");
    const Slot &sl = b->slots[slot];
    const size_t n = 9 * (size_t)sl.p.nx * sl.p.ny;
    void *cur = slot_pop(sl, (int)(b->h_dyn[slot].t & 1));
    if (on_device) {
        BCK(b, b->ops->get_pop(cur, sl.gd, sl.k, f, b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        return LBM_OK;
    }
    void *tmp = nullptr;
    BCK(b, cudaMallocAsync(&tmp, n * sizeof(double), b->stream));
    cudaError_t e = b->ops->get_pop(cur, sl.gd, sl.k, static_cast<double *>(tmp), b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    cudaFreeAsync(tmp, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("populations: ") + cudaGetErrorString(e));
    return LBM_OK;
}

}  // extern "C"
