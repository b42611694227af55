// prc_ops_impl.cuh -- host launchers of the kernels for one storage type.
// Included once by each of ops_f64.cu / ops_f32.cu / ops_f16.cu with
// PRC_S (storage type), PRC_T (collision type) and PRC_OPS (table name).
#pragma once

#include "prc_ops.h"

namespace prc {
namespace {

using S = PRC_S;
using T = PRC_T;

struct TmaArgs {
    const CUtensorMap *tsrc, *tdst;
    const S *a;
    S *b;
    Coef<F2> k;
    Coef<float> kf;
    float *sn;
    double2 *partials;
    DevStatus *st;
    int rev;  // tile order of this step
};

template <int W, int H, int THREADS, int MINB, bool DRHO, bool EPI, bool FORCE>
cudaError_t launch_tma_t(const TmaArgs &x, const Plan &pl, const Grid &gd, cudaStream_t s)
{
    using Cf = TmaCfg<S, W, H, THREADS>;
    k_step_tma<S, W, H, THREADS, MINB, DRHO, EPI, FORCE><<<pl.n_int_ctas, THREADS, Cf::SMEM, s>>>(
        *x.tsrc, *x.tdst, x.a, x.b, gd, x.k, x.kf, x.sn, x.partials, x.st, Interior{pl.in.ix0, pl.in.iy0, pl.in.ntx,
        pl.in.nty, pl.in.xlast, pl.in.ylast, x.rev}, pl.edge);
    return cudaGetLastError();
}

template <int W, int H, int THREADS, int MINB, bool DRHO, bool EPI>
cudaError_t launch_tma_f(const TmaArgs &x, const Plan &pl, const Grid &gd, bool force, cudaStream_t s)
{
    if (force) return launch_tma_t<W, H, THREADS, MINB, DRHO, EPI, true>(x, pl, gd, s);
    return launch_tma_t<W, H, THREADS, MINB, DRHO, EPI, false>(x, pl, gd, s);
}

template <int W, int H, int THREADS, int MINB>
cudaError_t launch_tma(const CUtensorMap *tsrc, const CUtensorMap *tdst, const void *src, void *dst, const Plan &pl,
                       const Grid &gd,
                       const Coef<double> &kd, void *snap, double2 *partials, DevStatus *st, bool drho, bool epi,
                       bool force, int rev, cudaStream_t s)
{
    const TmaArgs x{tsrc, tdst, static_cast<const S *>(src), static_cast<S *>(dst), cast_coef<F2>(kd),
                    cast_coef<float>(kd), static_cast<float *>(snap), partials, st, rev};
    if (drho) {
        if (epi) return launch_tma_f<W, H, THREADS, MINB, true, true>(x, pl, gd, force, s);
        return launch_tma_f<W, H, THREADS, MINB, true, false>(x, pl, gd, force, s);
    }
    if (epi) return launch_tma_f<W, H, THREADS, MINB, false, true>(x, pl, gd, force, s);
    return launch_tma_f<W, H, THREADS, MINB, false, false>(x, pl, gd, force, s);
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
cudaError_t launch_general(const S *a, S *b, const Plan &pl, const Grid &gd, const Coef<double> &kd, T *sn,
                           double2 *partials, const DevStatus *st, cudaStream_t s)
{
    if constexpr (std::is_same<T, float>::value) {  // pair tile body, 64 x 8 tiles
        const Coef<float> kf = cast_coef<float>(kd);
        const Coef<F2> k2 = cast_coef<F2>(kd);
        if (gd.model == 1)
            k_step_pair<S, DRHO, EPI, FORCE, true><<<pl.n_edge_ctas, 256, 0, s>>>(a, b, gd, kf, k2, sn, partials, st,
                                                                                 pl.edge, pl.n_int_ctas);
        else
            k_step_pair<S, DRHO, EPI, FORCE, false><<<pl.n_edge_ctas, 256, 0, s>>>(a, b, gd, kf, k2, sn, partials,
                                                                                  st, pl.edge, pl.n_int_ctas);
        return cudaGetLastError();
    }
    const Coef<T> k = cast_coef<T>(kd);
    if (gd.model == 1)
        k_step<S, T, DRHO, EPI, FORCE, true><<<pl.n_edge_ctas, dim3(BX, BY), 0, s>>>(a, b, gd, k, sn, partials, st,
                                                                                     pl.edge, pl.n_int_ctas);
    else
        k_step<S, T, DRHO, EPI, FORCE, false><<<pl.n_edge_ctas, dim3(BX, BY), 0, s>>>(a, b, gd, k, sn, partials, st,
                                                                                      pl.edge, pl.n_int_ctas);
    return cudaGetLastError();
}

template <bool DRHO, bool EPI>
cudaError_t general_f(const S *a, S *b, const Plan &pl, const Grid &gd, const Coef<double> &k, T *sn, double2 *partials,
                      const DevStatus *st, bool force, cudaStream_t s)
{
    if (force) return launch_general<DRHO, EPI, true>(a, b, pl, gd, k, sn, partials, st, s);
    return launch_general<DRHO, EPI, false>(a, b, pl, gd, k, sn, partials, st, s);
}

cudaError_t op_step_general(const void *src, void *dst, const Plan &pl, const Grid &gd, const Coef<double> &kd,
                            void *snap, double2 *partials, const DevStatus *st, bool drho, bool epi, bool force,
                            cudaStream_t s)
{
    const S *a = static_cast<const S *>(src);
    S *b = static_cast<S *>(dst);
    T *sn = static_cast<T *>(snap);
    if (drho) {
        if (epi) return general_f<true, true>(a, b, pl, gd, kd, sn, partials, st, force, s);
        return general_f<true, false>(a, b, pl, gd, kd, sn, partials, st, force, s);
    }
    if (epi) return general_f<false, true>(a, b, pl, gd, kd, sn, partials, st, force, s);
    return general_f<false, false>(a, b, pl, gd, kd, sn, partials, st, force, s);
}

void op_coef_convert(const Coef<double> &in, void *out)
{
    BatchCoef<T> *c = static_cast<BatchCoef<T> *>(out);
    c->k = cast_coef<T>(in);
    c->k2 = cast_coef<F2>(in);
}

// resident CTAs per SM of both forms of the batch kernel (the smaller)
cudaError_t op_batch_occupancy(int *blocks_per_sm)
{
    int a = 0, c = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch<S, T, 0>, BX * BY, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_batch<S, T, 1>, BX * BY, 0);
    *blocks_per_sm = a < c ? a : c;
    return e;
}

// one cooperative launch (all CTAs co-resident, as the grid barrier needs)
cudaError_t op_batch_launch(const BatchInst *inst, const void *coefs, BatchDyn *dyn, int ninst, int total_tiles,
                            double2 *partials, BatchCtl *ctl, int steps, int grid, int spec, cudaStream_t s)
{
    const BatchCoef<T> *cf = static_cast<const BatchCoef<T> *>(coefs);
    void *args[] = {(void *)&inst, (void *)&cf, (void *)&dyn, (void *)&ninst, (void *)&total_tiles,
                    (void *)&partials, (void *)&ctl, (void *)&steps};
    const void *k = spec ? (const void *)k_batch<S, T, 1> : (const void *)k_batch<S, T, 0>;
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(BX, BY), args, 0, s);
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

cudaError_t op_add_rest(void *pop, const Grid &gd, const Coef<double> &k, double delta, cudaStream_t s)
{
    k_add_rest<S, T><<<row_grid(gd), 128, 0, s>>>(static_cast<S *>(pop), gd, k, delta);
    return cudaGetLastError();
}

template <bool DRHO, bool FORCE, bool RAW>
cudaError_t cluster_cfg_launch(const S *p0, const S *p1, const Grid &gd, const Coef<T> &k, const Coef<F2> &k2,
                               T *snap, DevStatus *st,
                               long long t0, int n, int nc, int rpc, int smem, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc, 1, 1);
    cfg.blockDim = dim3(CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const bool one = std::is_same<T, float>::value && rpc * ((gd.nx + 1) / 2) <= CL_THREADS;
    if constexpr (std::is_same<T, float>::value) {
        if (one)
            return cudaLaunchKernelEx(&cfg, k_cluster<S, T, DRHO, FORCE, RAW, true>, p0, p1, gd, k, k2, snap, st, t0,
                                      n, rpc);
    }
    return cudaLaunchKernelEx(&cfg, k_cluster<S, T, DRHO, FORCE, RAW, false>, p0, p1, gd, k, k2, snap, st, t0, n, rpc);
}

cudaError_t cluster_attr_one(const void *kern, int smem)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <bool DRHO, bool FORCE, bool RAW>
cudaError_t cluster_attr(int smem)
{
    cudaError_t e = cluster_attr_one((const void *)k_cluster<S, T, DRHO, FORCE, RAW, false>, smem);
    if (e != cudaSuccess) return e;
    if constexpr (std::is_same<T, float>::value)
        e = cluster_attr_one((const void *)k_cluster<S, T, DRHO, FORCE, RAW, true>, smem);
    return e;
}

template <bool RAW>
cudaError_t cluster_prepare_m(int smem)
{
    cudaError_t e;
    if ((e = cluster_attr<false, false, RAW>(smem)) != cudaSuccess) return e;
    if ((e = cluster_attr<false, true, RAW>(smem)) != cudaSuccess) return e;
    if ((e = cluster_attr<true, false, RAW>(smem)) != cudaSuccess) return e;
    return cluster_attr<true, true, RAW>(smem);
}

cudaError_t op_cluster_prepare(int smem)
{
    cudaError_t e = cluster_prepare_m<false>(smem);
    if (e != cudaSuccess) return e;
    return cluster_prepare_m<true>(smem);
}

cudaError_t op_cluster_max_active(int nc, int smem, int *n)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc, 1, 1);
    cfg.blockDim = dim3(CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(n, (void *)k_cluster<S, T, true, false, false, false>, &cfg);
}

cudaError_t op_cluster_launch(const void *pop0, const void *pop1, const Grid &gd, const Coef<double> &kd, void *snap,
                              DevStatus *st, long long t0, int n, int nc, int rpc, int smem, bool drho, bool force,
                              cudaStream_t s)
{
    const Coef<T> k = cast_coef<T>(kd);
    const Coef<F2> k2 = cast_coef<F2>(kd);
    const S *a = static_cast<const S *>(pop0), *b = static_cast<const S *>(pop1);
    T *sn = static_cast<T *>(snap);
    if (gd.model == 1) {
        if (drho) {
            if (force) return cluster_cfg_launch<true, true, true>(a, b, gd, k, k2, sn, st, t0, n, nc, rpc, smem, s);
            return cluster_cfg_launch<true, false, true>(a, b, gd, k, k2, sn, st, t0, n, nc, rpc, smem, s);
        }
        if (force) return cluster_cfg_launch<false, true, true>(a, b, gd, k, k2, sn, st, t0, n, nc, rpc, smem, s);
        return cluster_cfg_launch<false, false, true>(a, b, gd, k, k2, sn, st, t0, n, nc, rpc, smem, s);
    }
    if (drho) {
        if (force) return cluster_cfg_launch<true, true, false>(a, b, gd, k, k2, sn, st, t0, n, nc, rpc, smem, s);
        return cluster_cfg_launch<true, false, false>(a, b, gd, k, k2, sn, st, t0, n, nc, rpc, smem, s);
    }
    if (force) return cluster_cfg_launch<false, true, false>(a, b, gd, k, k2, sn, st, t0, n, nc, rpc, smem, s);
    return cluster_cfg_launch<false, false, false>(a, b, gd, k, k2, sn, st, t0, n, nc, rpc, smem, s);
}

template <typename TT>
cudaError_t op_batch_tma_prepare()
{
    if constexpr (std::is_same<TT, float>::value)
        return cudaFuncSetAttribute(k_batch_tma<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_tma_smem<S>());
    return cudaErrorNotSupported;
}

template <typename TT>
cudaError_t op_batch_tma_occupancy(int *blocks_per_sm)
{
    if constexpr (std::is_same<TT, float>::value)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_tma<S>, BT_THREADS,
                                                             batch_tma_smem<S>());
    *blocks_per_sm = 0;
    return cudaErrorNotSupported;
}

template <typename TT>
cudaError_t op_batch_tma_launch(const BatchInst *inst, const void *coefs, BatchDyn *dyn, int ninst, int tiles,
                                double2 *partials, BatchCtl *ctl, int steps, int grid, cudaStream_t s)
{
    if constexpr (std::is_same<TT, float>::value) {
        const BatchCoef<float> *cf = static_cast<const BatchCoef<float> *>(coefs);
        void *args[] = {(void *)&inst, (void *)&cf, (void *)&dyn, (void *)&ninst, (void *)&tiles, (void *)&partials,
                        (void *)&ctl, (void *)&steps};
        return cudaLaunchCooperativeKernel((const void *)k_batch_tma<S>, dim3(grid), dim3(BT_THREADS), args,
                                           batch_tma_smem<S>(), s);
    }
    return cudaErrorNotSupported;
}

}  // namespace

#define PRC_VARIANT(W, H, THREADS, MINB) \
    { W, H, THREADS, MINB, prepare_tma<W, H, THREADS, MINB>, launch_tma<W, H, THREADS, MINB> }

const DtypeOps PRC_OPS = {sizeof(S), sizeof(T), 16 / (int)sizeof(S), PRC_NVARIANTS, {PRC_VARIANTS},
                          op_step_general, sizeof(BatchCoef<T>), op_coef_convert, op_batch_occupancy, op_batch_launch,
                          op_init_fields, op_fields, op_set_pop, op_get_pop, op_mass_partial, op_add_rest,
                          op_cluster_prepare, op_cluster_max_active, op_cluster_launch,
                          std::is_same<T, float>::value ? op_batch_tma_prepare<T> : nullptr,
                          std::is_same<T, float>::value ? op_batch_tma_occupancy<T> : nullptr,
                          std::is_same<T, float>::value ? op_batch_tma_launch<T> : nullptr};

}  // namespace prc
