// Self-test of the bounded device waits (the staged step kernel's mbarrier
// waits): one warp waits on an mbarrier that nothing arrives on -- no copy is
// ever issued to it -- for a given number of polls, gives up, records the
// timeout in a status word and returns, exactly as the step kernel does when
// its copies do not land.  The host then reads LBM_E_TIMEOUT and the context
// stays usable.  The paper has no counterpart; this exercises failure
// reporting without faulting or hanging the device.
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

__global__ void __launch_bounds__(32) wait_selftest_kernel(long long polls, unsigned* status) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned FULL = 0xffffffffu;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // one arrival would complete phase 0; none comes
    mbar_init_fence();
  }
  __syncwarp();
  bool ok = false;
  for (long long it = 0; it < polls && !ok; ++it) ok = __any_sync(FULL, mbar_try_wait(&bar, 0));
  if (threadIdx.x == 0) *status = ok ? 0u : kStatusTimeout;
}

}  // namespace lbm

extern "C" lbm_status lbm_selftest_wait_timeout(int device, long long polls, int* result) {
  if (!result || polls < 1 || polls > (1ll << 20)) return LBM_E_INVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return LBM_E_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return LBM_E_CUDA;
  unsigned* d_status = nullptr;
  unsigned h = ~0u;
  lbm_status st = LBM_OK;
  if (cudaMalloc(&d_status, sizeof(unsigned)) != cudaSuccess) {
    st = LBM_E_NOMEM;
  } else {
    lbm::wait_selftest_kernel<<<1, 32>>>(polls, d_status);
    lbm::count_launches(1);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(&h, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = LBM_E_CUDA;
    cudaFree(d_status);
  }
  if (st == LBM_OK) *result = (h & lbm::kStatusTimeout) ? LBM_E_TIMEOUT : LBM_OK;
  if (prev != device) cudaSetDevice(prev);
  return st;
}
