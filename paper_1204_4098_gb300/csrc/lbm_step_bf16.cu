// Fused step, observe, state and mass kernels for StoreBF16 storage.
#include "lbm_launch.cuh"

LBM_DEFINE_PRECISION(bf16, lbm::StoreBF16)
