// prc_ops.h -- internal interface between the C ABI (lbm_api.cu) and the
// per-storage-type kernel translation units (ops_f64.cu, ops_f32.cu,
// ops_f16.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "prc_batch.cuh"
#include "prc_batch_tma.cuh"
#include "prc_cluster.cuh"
#include "prc_kernels.cuh"
#include "prc_tma.cuh"

namespace prc {

template <typename T>
inline Coef<T> cast_coef(const Coef<double> &d)
{
    Coef<T> c;
    const double *s = reinterpret_cast<const double *>(&d);
    T *o = reinterpret_cast<T *>(&c);
    for (size_t i = 0; i < sizeof(Coef<double>) / sizeof(double); i++) o[i] = from_double<T>(s[i]);
    return c;
}

// How one time step is split between the TMA interior kernel and the general
// (wall-aware) kernel on the remaining edge strips.
struct Plan {
    int tma;           // interior kernel in use
    Interior in;
    int n_int_ctas;    // persistent grid of the interior kernel; partials [0, n_int_ctas)
    Rects edge;        // rectangles of the general tile body (edge strips ride in the
                       // interior launch when tma != 0)
    int n_edge_ctas;   // general-kernel CTAs: partials [n_int_ctas, n_int_ctas + n_edge_ctas)
    int nparts;
};

constexpr int MAX_INTERIOR_CTAS = 1024;
constexpr int MAX_VARIANTS = 5;

// One compiled configuration of the interior kernel.
struct Variant {
    int w, h;         // tile (nodes)
    int threads;      // CTA size
    int ctas_per_sm;  // resident CTAs per SM (shared memory / register budget)
    cudaError_t (*prepare)();
    // tsrc: load descriptor of the source set (box = tile + ring); tdst:
    // store descriptor of the destination set (box = tile)
    // rev: take the interior tiles in reverse order (alternate steps)
    cudaError_t (*launch)(const CUtensorMap *tsrc, const CUtensorMap *tdst, const void *src, void *dst, const Plan &pl,
                          const Grid &gd, const Coef<double> &k, void *snap, double2 *partials, DevStatus *st,
                          bool drho, bool epi, bool force, int rev, cudaStream_t s);
};

struct DtypeOps {
    size_t elem;       // bytes per stored population
    size_t snap_elem;  // bytes per snapshot value (collision precision)
    int tma_padx;      // 16-byte alignment of the TMA x origin, in elements
    int nvariants;     // interior-kernel variants (0: general kernel only)
    Variant variants[MAX_VARIANTS];
    // general kernel on the rectangles of the plan (edge strips)
    cudaError_t (*step_general)(const void *src, void *dst, const Plan &pl, const Grid &gd, const Coef<double> &k,
                                void *snap, double2 *partials, const DevStatus *st, bool drho, bool epi, bool force,
                                cudaStream_t s);
    // batch: per-slot coefficient conversion, occupancy and the persistent launch
    size_t coef_bytes;
    void (*coef_convert)(const Coef<double> &in, void *out);
    cudaError_t (*batch_occupancy)(int *blocks_per_sm);
    // spec != 0: every instance has the density-gradient terms, no force and
    // the central-moment scheme (the specialised kernel)
    cudaError_t (*batch_launch)(const BatchInst *inst, const void *coefs, BatchDyn *dyn, int ninst, int total_tiles,
                                double2 *partials, BatchCtl *ctl, int steps, int grid, int spec, cudaStream_t s);
    cudaError_t (*init_fields)(void *dst, const Grid &gd, const Coef<double> &k, double gamma, const double *rho,
                               const double *ux, const double *uy, void *snap, cudaStream_t s);
    cudaError_t (*fields)(const void *src, const Grid &gd, const Coef<double> &k, double *rho, double *ux,
                          double *uy, void *snap, cudaStream_t s);
    cudaError_t (*set_pop)(void *dst, const Grid &gd, const Coef<double> &k, const double *f, cudaStream_t s);
    cudaError_t (*get_pop)(const void *src, const Grid &gd, const Coef<double> &k, double *f, cudaStream_t s);
    cudaError_t (*mass_partial)(const void *src, const Grid &gd, double2 *partials, cudaStream_t s);
    cudaError_t (*add_rest)(void *pop, const Grid &gd, const Coef<double> &k, double delta, cudaStream_t s);
    // cluster-resident engine: shared-memory / cluster-size opt-in, how many
    // clusters of nc CTAs with `smem` bytes fit at once (0: not launchable),
    // and one launch of n steps from the state after step t0
    cudaError_t (*cluster_prepare)(int smem);
    cudaError_t (*cluster_max_active)(int nc, int smem, int *n);
    cudaError_t (*cluster_launch)(const void *pop0, const void *pop1, const Grid &gd, const Coef<double> &k,
                                  void *snap, DevStatus *st, long long t0, int n, int nc, int rpc, int smem,
                                  bool drho, bool force, cudaStream_t s);
    // batch engine with TMA-staged tiles (k_batch_tma; FP32 / FP16
    // storage, null for FP64): shared-memory opt-in (once, outside any stream
    // capture), resident CTAs per SM, one cooperative launch
    cudaError_t (*batch_tma_prepare)();
    cudaError_t (*batch_tma_occupancy)(int *blocks_per_sm);
    cudaError_t (*batch_tma_launch)(const BatchInst *inst, const void *coefs, BatchDyn *dyn, int ninst, int tiles,
                                    double2 *partials, BatchCtl *ctl, int steps, int grid, cudaStream_t s);
};

extern const DtypeOps ops_f64, ops_f32, ops_f16;

// grid of the tiled kernels
inline dim3 step_grid(const Grid &gd) { return dim3((gd.nx + 31) / 32, (gd.ny + 7) / 8, 1); }

}  // namespace prc
