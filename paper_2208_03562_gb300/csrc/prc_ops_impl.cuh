// prc_ops_impl.cuh -- host launchers of the kernels for one storage type.
// Included once by each of ops_f64.cu / ops_f32.cu / ops_f16.cu with
// PRC_S (storage type), PRC_T (collision type) and PRC_OPS (table name).
#pragma once

#include "prc_ops.h"

namespace prc {
namespace {

using S = PRC_S;
using T = PRC_T;

template <int W, int H, int THREADS, int MINB, bool DRHO, bool EPI, bool FORCE>
cudaError_t launch_tma_t(const CUtensorMap *tsrc, S *b, const Plan &pl, const Grid &gd, const Coef<F2> &k,
                         float *sn, double2 *partials, DevStatus *st, cudaStream_t s)
{
    using Cf = TmaCfg<S, W, H, THREADS>;
    k_step_tma<S, W, H, THREADS, MINB, DRHO, EPI, FORCE><<<pl.n_int_ctas, THREADS, Cf::SMEM, s>>>(
        *tsrc, b, gd, k, sn, partials, st, pl.in);
    return cudaGetLastError();
}

template <int W, int H, int THREADS, int MINB, bool DRHO, bool EPI>
cudaError_t launch_tma_f(const CUtensorMap *tsrc, S *b, const Plan &pl, const Grid &gd, const Coef<F2> &k,
                         float *sn, double2 *partials, DevStatus *st, bool force, cudaStream_t s)
{
    if (force) return launch_tma_t<W, H, THREADS, MINB, DRHO, EPI, true>(tsrc, b, pl, gd, k, sn, partials, st, s);
    return launch_tma_t<W, H, THREADS, MINB, DRHO, EPI, false>(tsrc, b, pl, gd, k, sn, partials, st, s);
}

template <int W, int H, int THREADS, int MINB>
cudaError_t launch_tma(const CUtensorMap *tsrc, void *dst, const Plan &pl, const Grid &gd, const Coef<double> &kd,
                       void *snap, double2 *partials, DevStatus *st, bool drho, bool epi, bool force, cudaStream_t s)
{
    const Coef<F2> k = cast_coef<F2>(kd);
    S *b = static_cast<S *>(dst);
    float *sn = static_cast<float *>(snap);
    if (drho) {
        if (epi) return launch_tma_f<W, H, THREADS, MINB, true, true>(tsrc, b, pl, gd, k, sn, partials, st, force, s);
        return launch_tma_f<W, H, THREADS, MINB, true, false>(tsrc, b, pl, gd, k, sn, partials, st, force, s);
    }
    if (epi) return launch_tma_f<W, H, THREADS, MINB, false, true>(tsrc, b, pl, gd, k, sn, partials, st, force, s);
    return launch_tma_f<W, H, THREADS, MINB, false, false>(tsrc, b, pl, gd, k, sn, partials, st, force, s);
}

template <int W, int H, int THREADS, int MINB, bool DRHO, bool EPI, bool FORCE>
cudaError_t set_attr()
{
    return cudaFuncSetAttribute(k_step_tma<S, W, H, THREADS, MINB, DRHO, EPI, FORCE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, TmaCfg<S, W, H, THREADS>::SMEM);
}

// opt a variant's kernels into their dynamic shared memory (once, outside any
// stream capture)
template <int W, int H, int THREADS, int MINB>
cudaError_t prepare_tma()
{
    cudaError_t e;
    if ((e = set_attr<W, H, THREADS, MINB, false, false, false>()) != cudaSuccess) return e;
    if ((e = set_attr<W, H, THREADS, MINB, false, true, false>()) != cudaSuccess) return e;
    if ((e = set_attr<W, H, THREADS, MINB, true, false, false>()) != cudaSuccess) return e;
    if ((e = set_attr<W, H, THREADS, MINB, true, true, false>()) != cudaSuccess) return e;
    if ((e = set_attr<W, H, THREADS, MINB, false, false, true>()) != cudaSuccess) return e;
    if ((e = set_attr<W, H, THREADS, MINB, false, true, true>()) != cudaSuccess) return e;
    if ((e = set_attr<W, H, THREADS, MINB, true, false, true>()) != cudaSuccess) return e;
    return set_attr<W, H, THREADS, MINB, true, true, true>();
}

template <bool DRHO, bool EPI, bool FORCE>
cudaError_t launch_general(const S *a, S *b, const Plan &pl, const Grid &gd, const Coef<T> &k, T *sn,
                           double2 *partials, const DevStatus *st, cudaStream_t s)
{
    k_step<S, T, DRHO, EPI, FORCE><<<pl.n_edge_ctas, dim3(BX, BY), 0, s>>>(a, b, gd, k, sn, partials, st, pl.edge,
                                                                           pl.n_int_ctas);
    return cudaGetLastError();
}

template <bool DRHO, bool EPI>
cudaError_t general_f(const S *a, S *b, const Plan &pl, const Grid &gd, const Coef<T> &k, T *sn, double2 *partials,
                      const DevStatus *st, bool force, cudaStream_t s)
{
    if (force) return launch_general<DRHO, EPI, true>(a, b, pl, gd, k, sn, partials, st, s);
    return launch_general<DRHO, EPI, false>(a, b, pl, gd, k, sn, partials, st, s);
}

cudaError_t op_step_general(const void *src, void *dst, const Plan &pl, const Grid &gd, const Coef<double> &kd,
                            void *snap, double2 *partials, const DevStatus *st, bool drho, bool epi, bool force,
                            cudaStream_t s)
{
    const Coef<T> k = cast_coef<T>(kd);
    const S *a = static_cast<const S *>(src);
    S *b = static_cast<S *>(dst);
    T *sn = static_cast<T *>(snap);
    if (drho) {
        if (epi) return general_f<true, true>(a, b, pl, gd, k, sn, partials, st, force, s);
        return general_f<true, false>(a, b, pl, gd, k, sn, partials, st, force, s);
    }
    if (epi) return general_f<false, true>(a, b, pl, gd, k, sn, partials, st, force, s);
    return general_f<false, false>(a, b, pl, gd, k, sn, partials, st, force, s);
}

void op_coef_convert(const Coef<double> &in, void *out) { *static_cast<Coef<T> *>(out) = cast_coef<T>(in); }

cudaError_t op_batch_occupancy(int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch<S, T>, BX * BY, 0);
}

// one cooperative launch (all CTAs co-resident, as the grid barrier needs)
cudaError_t op_batch_launch(const BatchInst *inst, const void *coefs, BatchDyn *dyn, int ninst, int total_tiles,
                            double2 *partials, BatchCtl *ctl, int steps, int grid, cudaStream_t s)
{
    const Coef<T> *cf = static_cast<const Coef<T> *>(coefs);
    void *args[] = {(void *)&inst, (void *)&cf, (void *)&dyn, (void *)&ninst, (void *)&total_tiles,
                    (void *)&partials, (void *)&ctl, (void *)&steps};
    return cudaLaunchCooperativeKernel((const void *)k_batch<S, T>, dim3(grid), dim3(BX, BY), args, 0, s);
}

dim3 row_grid(const Grid &gd) { return dim3((gd.nx + 127) / 128, gd.ny, 1); }

cudaError_t op_init_fields(void *dst, const Grid &gd, const Coef<double> &k, double gamma, const double *rho,
                           const double *ux, const double *uy, void *snap, cudaStream_t s)
{
    k_init_fields<S, T><<<row_grid(gd), 128, 0, s>>>(static_cast<S *>(dst), gd, k, gamma, rho, ux, uy,
                                                     static_cast<T *>(snap));
    return cudaGetLastError();
}

cudaError_t op_fields(const void *src, const Grid &gd, const Coef<double> &k, double *rho, double *ux, double *uy,
                      void *snap, cudaStream_t s)
{
    k_fields<S, T><<<row_grid(gd), 128, 0, s>>>(static_cast<const S *>(src), gd, k, rho, ux, uy,
                                                static_cast<T *>(snap));
    return cudaGetLastError();
}

cudaError_t op_set_pop(void *dst, const Grid &gd, const Coef<double> &k, const double *f, cudaStream_t s)
{
    k_set_pop<S, T><<<row_grid(gd), 128, 0, s>>>(static_cast<S *>(dst), gd, k, f);
    return cudaGetLastError();
}

cudaError_t op_get_pop(const void *src, const Grid &gd, const Coef<double> &k, double *f, cudaStream_t s)
{
    k_get_pop<S, T><<<row_grid(gd), 128, 0, s>>>(static_cast<const S *>(src), gd, k, f);
    return cudaGetLastError();
}

cudaError_t op_mass_partial(const void *src, const Grid &gd, double2 *partials, cudaStream_t s)
{
    k_mass_partial<S, T><<<step_grid(gd), dim3(BX, BY), 0, s>>>(static_cast<const S *>(src), gd, partials);
    return cudaGetLastError();
}

}  // namespace

#define PRC_VARIANT(W, H, THREADS, MINB) \
    { W, H, THREADS, MINB, prepare_tma<W, H, THREADS, MINB>, launch_tma<W, H, THREADS, MINB> }

const DtypeOps PRC_OPS = {sizeof(S), sizeof(T), 16 / (int)sizeof(S), PRC_NVARIANTS, {PRC_VARIANTS},
                          op_step_general, sizeof(Coef<T>), op_coef_convert, op_batch_occupancy, op_batch_launch,
                          op_init_fields, op_fields, op_set_pop, op_get_pop, op_mass_partial};

}  // namespace prc
