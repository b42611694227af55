// ops_f64.cu -- kernels and launchers for double storage, double collision.
#define PRC_S double
#define PRC_T double
#define PRC_OPS ops_f64
#include "prc_ops_impl.cuh"
