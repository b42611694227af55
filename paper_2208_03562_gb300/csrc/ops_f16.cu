// ops_f16.cu -- kernels and launchers for __half storage, float collision.
#define PRC_S __half
#define PRC_T float
#define PRC_OPS ops_f16
#include "prc_ops_impl.cuh"
