// Fused step, observe, state and mass kernels for StoreF16 storage.
#include "lbm_launch.cuh"

LBM_DEFINE_PRECISION(f16, lbm::StoreF16)
