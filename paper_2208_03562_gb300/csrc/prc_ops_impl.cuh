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

template <bool DRHO, bool EPI, bool FORCE>
cudaError_t launch_tma(const CUtensorMap *tsrc, S *b, const Plan &pl, const Grid &gd, const Coef<F2> &k, float *sn,
                       double2 *partials, DevStatus *st, cudaStream_t s)
{
    if constexpr (TW > 0) {
        using Cf = TmaCfg<S, TW, TH>;
        k_step_tma<S, TW, TH, DRHO, EPI, FORCE><<<pl.n_int_ctas, Cf::THREADS, Cf::SMEM, s>>>(*tsrc, b, gd, k, sn,
                                                                                            partials, st, pl.in);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

template <bool DRHO, bool EPI, bool FORCE>
cudaError_t set_smem_attr()
{
    if constexpr (TW > 0) {
        return cudaFuncSetAttribute(k_step_tma<S, TW, TH, DRHO, EPI, FORCE>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, TmaCfg<S, TW, TH>::SMEM);
    }
    return cudaSuccess;
}

// opt the interior kernels into their dynamic shared memory (once, outside
// any stream capture)
cudaError_t op_prepare()
{
    cudaError_t e;
    if ((e = set_smem_attr<false, false, false>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<false, true, false>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<true, false, false>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<true, true, false>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<false, false, true>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<false, true, true>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<true, false, true>()) != cudaSuccess) return e;
    return set_smem_attr<true, true, true>();
}

template <bool DRHO, bool EPI, bool FORCE>
cudaError_t launch_general(const S *a, S *b, const Plan &pl, const Grid &gd, const Coef<T> &k, T *sn,
                           double2 *partials, const DevStatus *st, cudaStream_t s)
{
    k_step<S, T, DRHO, EPI, FORCE><<<pl.n_edge_ctas, dim3(BX, BY), 0, s>>>(a, b, gd, k, sn, partials, st, pl.edge,
                                                                           pl.n_int_ctas);
    return cudaGetLastError();
}

template <bool DRHO, bool EPI, bool FORCE>
cudaError_t step_both(const void *src, void *dst, const CUtensorMap *tsrc, const Plan &pl, const Grid &gd,
                      const Coef<double> &kd, void *snap, double2 *partials, DevStatus *st, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (pl.tma) {
        if constexpr (TW > 0)
            e = launch_tma<DRHO, EPI, FORCE>(tsrc, static_cast<S *>(dst), pl, gd, cast_coef<F2>(kd),
                                             static_cast<float *>(snap), partials, st, s);
        else
            e = cudaErrorNotSupported;
    }
    if (e == cudaSuccess && pl.n_edge_ctas > 0)
        e = launch_general<DRHO, EPI, FORCE>(static_cast<const S *>(src), static_cast<S *>(dst), pl, gd,
                                             cast_coef<T>(kd), static_cast<T *>(snap), partials, st, s);
    return e;
}

template <bool DRHO, bool EPI>
cudaError_t step_f(const void *src, void *dst, const CUtensorMap *tsrc, const Plan &pl, const Grid &gd,
                   const Coef<double> &kd, void *snap, double2 *partials, DevStatus *st, bool force, cudaStream_t s)
{
    if (force) return step_both<DRHO, EPI, true>(src, dst, tsrc, pl, gd, kd, snap, partials, st, s);
    return step_both<DRHO, EPI, false>(src, dst, tsrc, pl, gd, kd, snap, partials, st, s);
}

cudaError_t op_step(const void *src, void *dst, const CUtensorMap *tsrc, const Plan &pl, const Grid &gd,
                    const Coef<double> &kd, void *snap, double2 *partials, DevStatus *st, bool drho, bool epi,
                    bool force, cudaStream_t s)
{
    if (drho) {
        if (epi) return step_f<true, true>(src, dst, tsrc, pl, gd, kd, snap, partials, st, force, s);
        return step_f<true, false>(src, dst, tsrc, pl, gd, kd, snap, partials, st, force, s);
    }
    if (epi) return step_f<false, true>(src, dst, tsrc, pl, gd, kd, snap, partials, st, force, s);
    return step_f<false, false>(src, dst, tsrc, pl, gd, kd, snap, partials, st, force, s);
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
