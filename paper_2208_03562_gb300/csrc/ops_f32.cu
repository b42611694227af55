// ops_f32.cu -- kernels and launchers for float storage, float collision
// (interior TMA tile 64x32; 0 = general kernel only).
#define PRC_S float
#define PRC_T float
#define PRC_TMA_W 64
#define PRC_TMA_H 32
#define PRC_OPS ops_f32
#include "prc_ops_impl.cuh"
