// ops_f16.cu -- kernels and launchers for __half storage, float collision.
// Interior-kernel variants (tile w x h, CTA threads, CTAs per SM): PRC_VARIANT(128, 16, 512, 1), PRC_VARIANT(128, 8, 256, 2), PRC_VARIANT(64, 16, 256, 2), PRC_VARIANT(64, 32, 512, 1).
#define PRC_S __half
#define PRC_T float
#define PRC_OPS ops_f16
#define PRC_NVARIANTS 4
#define PRC_VARIANTS PRC_VARIANT(128, 16, 512, 1), PRC_VARIANT(128, 8, 256, 2), PRC_VARIANT(64, 16, 256, 2), PRC_VARIANT(64, 32, 512, 1)
#include "prc_ops_impl.cuh"
