// ops_f16.cu -- kernels and launchers for __half storage, float collision
// (interior TMA tile 128x32; 0 = general kernel only).
#define PRC_S __half
#define PRC_T float
#define PRC_TMA_W 128
#define PRC_TMA_H 32
#define PRC_OPS ops_f16
#include "prc_ops_impl.cuh"
