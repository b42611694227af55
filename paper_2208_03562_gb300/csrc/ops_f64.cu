// ops_f64.cu -- kernels and launchers for double storage, double collision
// (interior TMA tile 0x0; 0 = general kernel only).
#define PRC_S double
#define PRC_T double
#define PRC_TMA_W 0
#define PRC_TMA_H 0
#define PRC_OPS ops_f64
#include "prc_ops_impl.cuh"
