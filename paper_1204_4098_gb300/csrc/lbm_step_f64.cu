// Fused step, observe, state and mass kernels for StoreF64 storage.
#include "lbm_launch.cuh"

LBM_DEFINE_PRECISION(f64, lbm::StoreF64)
