// prc_ops_impl.cuh -- host launchers of the kernels for one storage type.
// Included once by each of ops_f64.cu / ops_f32.cu / ops_f16.cu with
// PRC_S (storage type), PRC_T (collision type) and PRC_OPS (table name).
#pragma once

#include "prc_kernels.cuh"
#include "prc_ops.h"

namespace prc {
namespace {

using S = PRC_S;
using T = PRC_T;

cudaError_t op_step(const void *src, void *dst, const Grid &gd, const Coef<double> &kd, void *snap,
                    double2 *partials, const DevStatus *st, bool drho, bool epi, cudaStream_t s)
{
    const Coef<T> k = cast_coef<T>(kd);
    const dim3 grid = step_grid(gd), block(BX, BY);
    const S *a = static_cast<const S *>(src);
    S *b = static_cast<S *>(dst);
    T *sn = static_cast<T *>(snap);
    if (drho) {
        if (epi) k_step<S, T, true, true><<<grid, block, 0, s>>>(a, b, gd, k, sn, partials, st);
        else k_step<S, T, true, false><<<grid, block, 0, s>>>(a, b, gd, k, sn, partials, st);
    } else {
        if (epi) k_step<S, T, false, true><<<grid, block, 0, s>>>(a, b, gd, k, sn, partials, st);
        else k_step<S, T, false, false><<<grid, block, 0, s>>>(a, b, gd, k, sn, partials, st);
    }
    return cudaGetLastError();
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

const DtypeOps PRC_OPS = {sizeof(S), sizeof(T), op_step, op_init_fields, op_fields, op_set_pop, op_get_pop,
                          op_mass_partial};

}  // namespace prc
