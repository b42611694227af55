// ops_f32.cu -- kernels and launchers for float storage, float collision.
#define PRC_S float
#define PRC_T float
#define PRC_OPS ops_f32
#include "prc_ops_impl.cuh"
