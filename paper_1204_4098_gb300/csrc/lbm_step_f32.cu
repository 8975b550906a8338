// Fused step, observe, state and mass kernels for StoreF32 storage.
#include "lbm_launch.cuh"

LBM_DEFINE_PRECISION(f32, lbm::StoreF32)
