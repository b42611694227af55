// ops_f32.cu -- kernels and launchers for float storage, float collision.
// Interior-kernel variants (tile w x h, CTA threads, CTAs per SM): PRC_VARIANT(64, 8, 256, 2), PRC_VARIANT(64, 16, 256, 2), PRC_VARIANT(64, 32, 512, 1), PRC_VARIANT(64, 16, 512, 1).
#define PRC_S float
#define PRC_T float
#define PRC_OPS ops_f32
#define PRC_NVARIANTS 4
#define PRC_VARIANTS PRC_VARIANT(64, 8, 256, 2), PRC_VARIANT(64, 16, 256, 2), PRC_VARIANT(64, 32, 512, 1), PRC_VARIANT(64, 16, 512, 1)
#include "prc_ops_impl.cuh"
