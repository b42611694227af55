// ops_f64.cu -- kernels and launchers for double storage, double collision.
// Interior-kernel variants (tile w x h, CTA threads, CTAs per SM): none.
#define PRC_S double
#define PRC_T double
#define PRC_OPS ops_f64
#define PRC_NVARIANTS 0
#define PRC_VARIANTS 
#include "prc_ops_impl.cuh"
