// Allocation-free FP64 sum of FP32 values (the mass of an FP32 population
// buffer), for callers that cannot call cudaMalloc.
//
// Who cannot allocate: code whose device memory is owned by another
// allocator (a framework's caching pool that has reserved the device, or a
// fixed memory budget), and code paths where cudaMalloc is not allowed or
// would synchronise the device at the wrong moment (latency-critical
// serving loops, stream-ordered code that must not block).  They pass their
// own input buffer and output slot; the partial sums live in a fixed,
// file-scope device array instead of a cudaMalloc'd scratch buffer.
//
// The paper has no counterpart; this is a deployment helper.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"

namespace {

constexpr int kMaxBlocks = 1024;                    // 8 KB of partial sums
constexpr size_t kMinPerBlock = 4096;               // values per block at least
constexpr size_t kMaxValues = size_t(1) << 30;      // largest accepted n
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Shared by every call on a device, and held by every GPU that loads the
// library until the process exits.  Each call overwrites the entries it
// uses, so nothing needs clearing between calls.
static __device__ __align__(256) double g_partial[kMaxBlocks];

std::mutex g_setup_mutex;
double* g_partial_addr[kMaxDevices] = {nullptr};

// Blocks of a call: enough to spread n over the GPU (one per kMinPerBlock
// values, at most kMaxBlocks).  Depends only on n.
int blocks_for(size_t n) {
  const size_t b = (n + kMinPerBlock - 1) / kMinPerBlock;
  return int(b < size_t(kMaxBlocks) ? b : size_t(kMaxBlocks));
}

// Block-wide sum.  The result is valid in thread 0 only (the other threads
// get 0); every launch of the kernels below uses exactly kThreads threads,
// which the shared array is sized for.
__device__ double block_reduce(double v, double* smem) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) smem[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) s += smem[i];
  return s;
}

// Block b of gridDim.x sums the contiguous range [b * per, min((b + 1) * per,
// n)), per = ceil(n / gridDim.x), in a fixed order into partial[b]: the
// ranges and the order depend only on n, so the result does not depend on
// scheduling.
__global__ void __launch_bounds__(kThreads)
range_sum_kernel(const float* __restrict__ x, size_t n, double* partial) {
  __shared__ double smem[kThreads / 32];
  const size_t per = (n + gridDim.x - 1) / gridDim.x;
  const size_t begin = size_t(blockIdx.x) * per;
  const size_t end = begin + per < n ? begin + per : n;
  double acc = 0.0;
  for (size_t i = begin + threadIdx.x; i < end; i += kThreads) acc += double(x[i]);
  const double s = block_reduce(acc, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads)
final_sum_kernel(const double* partial, int nblocks, double* out) {
  __shared__ double smem[kThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kThreads) acc += partial[i];
  const double s = block_reduce(acc, smem);
  if (threadIdx.x == 0) *out = s;
}

// Device address of g_partial on the current device, looked up once per
// device and cached for the life of the process.  In host code the name
// g_partial is only a host-side stand-in, so the address has to come from
// cudaGetSymbolAddress.  A device reset (cudaDeviceReset) reloads the
// module and makes the cached address stale; the entry point's contract
// excludes resetting a device it has been used on.
cudaError_t partial_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partial_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_partial);
    if (e != cudaSuccess) return e;
    g_partial_addr[dev] = p;
  }
  *out = g_partial_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_mass_f32_noalloc(const float* d_values, size_t n, double* d_out,
                                           void* cuda_stream) {
  if (!d_out || (n > 0 && !d_values)) return LBM_E_INVAL;
  if (n > kMaxValues) return LBM_E_INVAL;  // the documented maximum
  double* partial = nullptr;
  if (partial_address(&partial) != cudaSuccess) return LBM_E_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nblocks = blocks_for(n);
  if (nblocks > 0) range_sum_kernel<<<nblocks, kThreads, 0, s>>>(d_values, n, partial);
  final_sum_kernel<<<1, kThreads, 0, s>>>(partial, nblocks, d_out);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}
