// prc_ops_impl.cuh -- host launchers of the kernels for one storage type.
// Included once by each of ops_f64.cu / ops_f32.cu / ops_f16.cu with
// PRC_S (storage type), PRC_T (collision type) and PRC_OPS (table name).
#pragma once

#include "prc_ops.h"

namespace prc {
namespace {

using S = PRC_S;
using T = PRC_T;
constexpr int TW = PRC_TMA_W, TH = PRC_TMA_H;

template <bool DRHO, bool EPI>
cudaError_t launch_tma(const CUtensorMap *tsrc, S *b, const Plan &pl, const Grid &gd, const Coef<T> &k, T *sn,
                       double2 *partials, DevStatus *st, cudaStream_t s)
{
    if constexpr (TW > 0) {
        using Cf = TmaCfg<S, TW, TH>;
        k_step_tma<S, T, TW, TH, DRHO, EPI><<<pl.n_int_ctas, Cf::THREADS, Cf::SMEM, s>>>(*tsrc, b, gd, k, sn,
                                                                                        partials, st, pl.in);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

// opt the interior kernels into their dynamic shared memory (once, outside
// any stream capture)
cudaError_t op_prepare()
{
    if constexpr (TW > 0) {
        using Cf = TmaCfg<S, TW, TH>;
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_step_tma<S, T, TW, TH, false, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_step_tma<S, T, TW, TH, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_step_tma<S, T, TW, TH, true, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM)) != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_step_tma<S, T, TW, TH, true, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM);
    }
    return cudaSuccess;
}

template <bool DRHO, bool EPI>
cudaError_t launch_general(const S *a, S *b, const Plan &pl, const Grid &gd, const Coef<T> &k, T *sn,
                           double2 *partials, const DevStatus *st, cudaStream_t s)
{
    k_step<S, T, DRHO, EPI><<<pl.n_edge_ctas, dim3(BX, BY), 0, s>>>(a, b, gd, k, sn, partials, st, pl.edge,
                                                                    pl.n_int_ctas);
    return cudaGetLastError();
}

template <bool DRHO, bool EPI>
cudaError_t step_both(const void *src, void *dst, const CUtensorMap *tsrc, const Plan &pl, const Grid &gd,
                      const Coef<T> &k, T *sn, double2 *partials, DevStatus *st, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (pl.tma) e = launch_tma<DRHO, EPI>(tsrc, static_cast<S *>(dst), pl, gd, k, sn, partials, st, s);
    if (e == cudaSuccess && pl.n_edge_ctas > 0)
        e = launch_general<DRHO, EPI>(static_cast<const S *>(src), static_cast<S *>(dst), pl, gd, k, sn, partials,
                                      st, s);
    return e;
}

cudaError_t op_step(const void *src, void *dst, const CUtensorMap *tsrc, const Plan &pl, const Grid &gd,
                    const Coef<double> &kd, void *snap, double2 *partials, DevStatus *st, bool drho, bool epi,
                    cudaStream_t s)
{
    const Coef<T> k = cast_coef<T>(kd);
    T *sn = static_cast<T *>(snap);
    if (drho) {
        if (epi) return step_both<true, true>(src, dst, tsrc, pl, gd, k, sn, partials, st, s);
        return step_both<true, false>(src, dst, tsrc, pl, gd, k, sn, partials, st, s);
    }
    if (epi) return step_both<false, true>(src, dst, tsrc, pl, gd, k, sn, partials, st, s);
    return step_both<false, false>(src, dst, tsrc, pl, gd, k, sn, partials, st, s);
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

const DtypeOps PRC_OPS = {sizeof(S), sizeof(T), TW, TH, TW > 0 ? 16 / (int)sizeof(S) : 0,
                          op_prepare, op_step, op_init_fields, op_fields, op_set_pop, op_get_pop,
                          op_mass_partial};

}  // namespace prc
