// ops_f16.cu -- kernels and launchers for __half storage, float collision.
// Interior-kernel variants (tile w x h, CTA threads, CTAs per SM): PRC_VARIANT(128, 16, 512, 1), PRC_VARIANT(128, 8, 256, 2), PRC_VARIANT(64, 16, 256, 2), PRC_VARIANT(64, 32, 512, 1), PRC_VARIANT(64, 8, 256, 2).
// The last one has the tile shape of the batch engine's TMA-staged body, so a
// single handle can run exactly what a batch slot runs.
#define PRC_S __half
#define PRC_T float
#define PRC_OPS ops_f16
#define PRC_NVARIANTS 5
#define PRC_VARIANTS PRC_VARIANT(128, 16, 512, 1), PRC_VARIANT(128, 8, 256, 2), PRC_VARIANT(64, 16, 256, 2), PRC_VARIANT(64, 32, 512, 1), PRC_VARIANT(64, 8, 256, 2)
#include "prc_ops_impl.cuh"
