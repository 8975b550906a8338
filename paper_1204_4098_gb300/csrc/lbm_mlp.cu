// Warm-start network: a 4 -> 64 -> 64 -> 3 tanh MLP trained and evaluated
// by hand-written kernels.
//
//   h1 = tanh(x W1 + b1),  h2 = tanh(h1 W2 + b2),  y = h2 W3 + b3,
//   L  = mean over samples and outputs of (y - t)^2,  Adam updates.
//
// Parameters are one flat FP32 vector W1[4][64], b1[64], W2[64][64], b2[64],
// W3[64][3], b3[3] (4675 values).  Training runs as ONE launch of a single
// 128-thread CTA for all epochs: thread b carries sample b of the minibatch
// through the forward and backward pass (activations in shared memory), then
// every thread owns 37 parameters, sums their gradients over the minibatch
// and applies Adam with its moments held in registers.  The network is far
// too small for tensor cores or more SMs to matter.  The paper has no
// network; it serves the warm start of the parameter sweeps.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {

constexpr int kIn = 4, kHid = 64, kOut = 3;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kIn * kHid;    // 256
constexpr int kOffW2 = kOffB1 + kHid;          // 320
constexpr int kOffB2 = kOffW2 + kHid * kHid;   // 4416
constexpr int kOffW3 = kOffB2 + kHid;          // 4480
constexpr int kOffB3 = kOffW3 + kHid * kOut;   // 4672
constexpr int kNParams = kOffB3 + kOut;        // 4675
constexpr int kTrainThreads = 128;             // largest minibatch
constexpr int kOwn = (kNParams + kTrainThreads - 1) / kTrainThreads;  // 37
constexpr int kRow = kHid + 1;                 // padded activation row (no bank conflicts)

struct TrainSmem {
  float W[kNParams];
  float X[kTrainThreads * kIn];
  float T[kTrainThreads * kOut];
  float DY[kTrainThreads * kOut];
  float H1[kTrainThreads * kRow];
  float H2[kTrainThreads * kRow];
  float DZ1[kTrainThreads * kRow];
  float DZ2[kTrainThreads * kRow];
  float red[kTrainThreads / 32];
};

// Gradient of parameter p summed over the nb rows of the minibatch.
__device__ __forceinline__ float param_grad(const TrainSmem& s, int p, int nb) {
  float g = 0.f;
  if (p < kOffB1) {  // W1[i][j]
    const int i = p / kHid, j = p % kHid;
    for (int b = 0; b < nb; ++b) g = fmaf(s.X[b * kIn + i], s.DZ1[b * kRow + j], g);
  } else if (p < kOffW2) {
    const int j = p - kOffB1;
    for (int b = 0; b < nb; ++b) g += s.DZ1[b * kRow + j];
  } else if (p < kOffB2) {  // W2[i][j]
    const int q = p - kOffW2, i = q / kHid, j = q % kHid;
    for (int b = 0; b < nb; ++b) g = fmaf(s.H1[b * kRow + i], s.DZ2[b * kRow + j], g);
  } else if (p < kOffW3) {
    const int j = p - kOffB2;
    for (int b = 0; b < nb; ++b) g += s.DZ2[b * kRow + j];
  } else if (p < kOffB3) {  // W3[j][k]
    const int q = p - kOffW3, j = q / kOut, k = q % kOut;
    for (int b = 0; b < nb; ++b) g = fmaf(s.H2[b * kRow + j], s.DY[b * kOut + k], g);
  } else if (p < kNParams) {
    const int k = p - kOffB3;
    for (int b = 0; b < nb; ++b) g += s.DY[b * kOut + k];
  }
  return g;
}

// mode 0: train `epochs` epochs over `order` (epochs x n sample indices) with
// Adam; mode 1: one full-batch gradient of the first `n` samples (n <= 128)
// into grad_out, no update.  loss_out gets the last minibatch's loss.
__global__ void __launch_bounds__(kTrainThreads)
mlp_train_kernel(float* params, float* adam_m, float* adam_v, const float* __restrict__ X,
                 const float* __restrict__ Y, int n, const int* __restrict__ order, int epochs,
                 int batch, float lr, int t0, int mode, float* grad_out, float* loss_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int tid = threadIdx.x;
  for (int p = tid; p < kNParams; p += kTrainThreads) s.W[p] = params[p];
  float m[kOwn], v[kOwn];
#pragma unroll
  for (int k = 0; k < kOwn; ++k) {
    const int p = tid + k * kTrainThreads;
    m[k] = (mode == 0 && p < kNParams) ? adam_m[p] : 0.f;
    v[k] = (mode == 0 && p < kNParams) ? adam_v[p] : 0.f;
  }
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  float b1t = powf(beta1, float(t0)), b2t = powf(beta2, float(t0));
  const int per_epoch = (n + batch - 1) / batch;
  const int steps = mode == 0 ? epochs * per_epoch : 1;
  float last_loss = 0.f;
  __syncthreads();

  for (int st = 0; st < steps; ++st) {
    const int e = st / per_epoch, k0 = (st % per_epoch) * batch;
    const int nb = mode == 0 ? min(batch, n - k0) : n;
    // minibatch rows into shared memory
    if (tid < nb) {
      const int idx = mode == 0 ? order[size_t(e) * n + k0 + tid] : tid;
#pragma unroll
      for (int i = 0; i < kIn; ++i) s.X[tid * kIn + i] = X[size_t(idx) * kIn + i];
#pragma unroll
      for (int k = 0; k < kOut; ++k) s.T[tid * kOut + k] = Y[size_t(idx) * kOut + k];
    }
    __syncthreads();
    float sq = 0.f;
    if (tid < nb) {
      const int b = tid;
      float h1[kHid];
#pragma unroll
      for (int j = 0; j < kHid; ++j) {
        float z = s.W[kOffB1 + j];
#pragma unroll
        for (int i = 0; i < kIn; ++i) z = fmaf(s.X[b * kIn + i], s.W[kOffW1 + i * kHid + j], z);
        h1[j] = tanhf(z);
        s.H1[b * kRow + j] = h1[j];
      }
      float y[kOut];
#pragma unroll
      for (int k = 0; k < kOut; ++k) y[k] = s.W[kOffB3 + k];
      for (int j = 0; j < kHid; ++j) {
        float z = s.W[kOffB2 + j];
#pragma unroll
        for (int i = 0; i < kHid; ++i) z = fmaf(h1[i], s.W[kOffW2 + i * kHid + j], z);
        const float h = tanhf(z);
        s.H2[b * kRow + j] = h;
#pragma unroll
        for (int k = 0; k < kOut; ++k) y[k] = fmaf(h, s.W[kOffW3 + j * kOut + k], y[k]);
      }
      const float scale = 2.f / float(nb * kOut);
      float dy[kOut];
#pragma unroll
      for (int k = 0; k < kOut; ++k) {
        const float d = y[k] - s.T[b * kOut + k];
        sq = fmaf(d, d, sq);
        dy[k] = scale * d;
        s.DY[b * kOut + k] = dy[k];
      }
      float dz2[kHid];
#pragma unroll
      for (int j = 0; j < kHid; ++j) {
        float g = 0.f;
#pragma unroll
        for (int k = 0; k < kOut; ++k) g = fmaf(dy[k], s.W[kOffW3 + j * kOut + k], g);
        const float h = s.H2[b * kRow + j];
        dz2[j] = g * (1.f - h * h);
        s.DZ2[b * kRow + j] = dz2[j];
      }
      for (int i = 0; i < kHid; ++i) {
        float g = 0.f;
#pragma unroll
        for (int j = 0; j < kHid; ++j) g = fmaf(dz2[j], s.W[kOffW2 + i * kHid + j], g);
        const float h = s.H1[b * kRow + i];
        s.DZ1[b * kRow + i] = g * (1.f - h * h);
      }
    }
    // minibatch loss
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if ((tid & 31) == 0) s.red[tid >> 5] = sq;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < kTrainThreads / 32; ++w) t += s.red[w];
      last_loss = t / float(nb * kOut);
    }
    // gradients of the owned parameters, then Adam
    b1t *= beta1;
    b2t *= beta2;
#pragma unroll
    for (int k = 0; k < kOwn; ++k) {
      const int p = tid + k * kTrainThreads;
      if (p < kNParams) {
        const float g = param_grad(s, p, nb);
        if (mode == 1) {
          grad_out[p] = g;
        } else {
          m[k] = fmaf(beta1, m[k], (1.f - beta1) * g);
          v[k] = fmaf(beta2, v[k], (1.f - beta2) * g * g);
          const float mh = m[k] / (1.f - b1t), vh = v[k] / (1.f - b2t);
          s.W[p] -= lr * mh / (sqrtf(vh) + eps);
        }
      }
    }
    __syncthreads();
  }
  for (int p = tid; p < kNParams; p += kTrainThreads) params[p] = s.W[p];
#pragma unroll
  for (int k = 0; k < kOwn; ++k) {
    const int p = tid + k * kTrainThreads;
    if (mode == 0 && p < kNParams) {
      adam_m[p] = m[k];
      adam_v[p] = v[k];
    }
  }
  if (tid == 0 && loss_out) *loss_out = last_loss;
}

// y = network(x), one thread per sample.
__global__ void __launch_bounds__(256)
mlp_predict_kernel(const float* __restrict__ params, const float* __restrict__ X, int n,
                   float* Y) {
  __shared__ float W[kNParams];
  for (int p = threadIdx.x; p < kNParams; p += blockDim.x) W[p] = params[p];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  float x[kIn], h1[kHid], y[kOut];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = X[size_t(b) * kIn + i];
#pragma unroll
  for (int j = 0; j < kHid; ++j) {
    float z = W[kOffB1 + j];
#pragma unroll
    for (int i = 0; i < kIn; ++i) z = fmaf(x[i], W[kOffW1 + i * kHid + j], z);
    h1[j] = tanhf(z);
  }
#pragma unroll
  for (int k = 0; k < kOut; ++k) y[k] = W[kOffB3 + k];
  for (int j = 0; j < kHid; ++j) {
    float z = W[kOffB2 + j];
#pragma unroll
    for (int i = 0; i < kHid; ++i) z = fmaf(h1[i], W[kOffW2 + i * kHid + j], z);
    const float h = tanhf(z);
#pragma unroll
    for (int k = 0; k < kOut; ++k) y[k] = fmaf(h, W[kOffW3 + j * kOut + k], y[k]);
  }
#pragma unroll
  for (int k = 0; k < kOut; ++k) Y[size_t(b) * kOut + k] = y[k];
}

}  // namespace lbm

using namespace lbm;

struct lbm_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float* d_params = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_scratch = nullptr;  // gradient / loss
  int adam_t = 0;
  std::string err;
};

namespace {

lbm_status mfail(lbm_mlp* m, lbm_status st, const std::string& msg) {
  if (m) m->err = msg;
  return st;
}

#define LBM_MCUDA(m, call)                                                               \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return mfail(m, LBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

struct MDeviceGuard {
  int prev = -1;
  explicit MDeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~MDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Copies n host floats into a temporary device buffer.
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

}  // namespace

extern "C" {

int lbm_mlp_num_params(void) { return kNParams; }

lbm_status lbm_mlp_create(int device, void* cuda_stream, lbm_mlp** out) {
  if (!out) return LBM_E_INVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LBM_E_CUDA;
  MDeviceGuard guard(device);
  lbm_mlp* m = new lbm_mlp();
  m->device = device;
  if (cuda_stream) {
    m->stream = static_cast<cudaStream_t>(cuda_stream);
  } else if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) == cudaSuccess) {
    m->own_stream = true;
  } else {
    delete m;
    return LBM_E_CUDA;
  }
  bool ok = cudaMalloc(&m->d_params, kNParams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->d_m, kNParams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->d_v, kNParams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->d_scratch, (kNParams + 1) * sizeof(float)) == cudaSuccess &&
            cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(sizeof(TrainSmem))) == cudaSuccess &&
            cudaMemsetAsync(m->d_params, 0, kNParams * sizeof(float), m->stream) == cudaSuccess &&
            cudaMemsetAsync(m->d_m, 0, kNParams * sizeof(float), m->stream) == cudaSuccess &&
            cudaMemsetAsync(m->d_v, 0, kNParams * sizeof(float), m->stream) == cudaSuccess &&
            cudaStreamSynchronize(m->stream) == cudaSuccess;
  if (!ok) {
    lbm_mlp_destroy(m);
    return LBM_E_NOMEM;
  }
  *out = m;
  return LBM_OK;
}

lbm_status lbm_mlp_destroy(lbm_mlp* m) {
  if (!m) return LBM_OK;
  MDeviceGuard guard(m->device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  cudaFree(m->d_params);
  cudaFree(m->d_m);
  cudaFree(m->d_v);
  cudaFree(m->d_scratch);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
  delete m;
  return LBM_OK;
}

const char* lbm_mlp_last_error(const lbm_mlp* m) { return m ? m->err.c_str() : ""; }

lbm_status lbm_mlp_set_params(lbm_mlp* m, const float* params) {
  if (!m || !params) return mfail(m, LBM_E_INVAL, "null argument");
  MDeviceGuard guard(m->device);
  LBM_MCUDA(m, cudaMemcpyAsync(m->d_params, params, kNParams * sizeof(float),
                               cudaMemcpyHostToDevice, m->stream));
  LBM_MCUDA(m, cudaMemsetAsync(m->d_m, 0, kNParams * sizeof(float), m->stream));
  LBM_MCUDA(m, cudaMemsetAsync(m->d_v, 0, kNParams * sizeof(float), m->stream));
  LBM_MCUDA(m, cudaStreamSynchronize(m->stream));
  m->adam_t = 0;
  return LBM_OK;
}

lbm_status lbm_mlp_get_params(lbm_mlp* m, float* params) {
  if (!m || !params) return mfail(m, LBM_E_INVAL, "null argument");
  MDeviceGuard guard(m->device);
  LBM_MCUDA(m, cudaMemcpyAsync(params, m->d_params, kNParams * sizeof(float),
                               cudaMemcpyDeviceToHost, m->stream));
  LBM_MCUDA(m, cudaStreamSynchronize(m->stream));
  return LBM_OK;
}

lbm_status lbm_mlp_gradient(lbm_mlp* m, const float* X, const float* Y, int n, float* grad,
                            float* loss) {
  if (!m || !X || !Y || !grad || n < 1 || n > kTrainThreads)
    return mfail(m, LBM_E_INVAL, "need 1 <= n <= 128 and non-null arrays");
  MDeviceGuard guard(m->device);
  DevBuf dx, dy;
  LBM_MCUDA(m, cudaMalloc(&dx.p, size_t(n) * kIn * sizeof(float)));
  LBM_MCUDA(m, cudaMalloc(&dy.p, size_t(n) * kOut * sizeof(float)));
  LBM_MCUDA(m, cudaMemcpyAsync(dx.p, X, size_t(n) * kIn * sizeof(float), cudaMemcpyHostToDevice,
                               m->stream));
  LBM_MCUDA(m, cudaMemcpyAsync(dy.p, Y, size_t(n) * kOut * sizeof(float), cudaMemcpyHostToDevice,
                               m->stream));
  mlp_train_kernel<<<1, kTrainThreads, sizeof(TrainSmem), m->stream>>>(
      m->d_params, m->d_m, m->d_v, static_cast<float*>(dx.p), static_cast<float*>(dy.p), n,
      nullptr, 1, n, 0.f, m->adam_t, 1, m->d_scratch, m->d_scratch + kNParams);
  LBM_MCUDA(m, cudaGetLastError());
  count_launches(1);
  LBM_MCUDA(m, cudaMemcpyAsync(grad, m->d_scratch, kNParams * sizeof(float),
                               cudaMemcpyDeviceToHost, m->stream));
  float l = 0.f;
  LBM_MCUDA(m, cudaMemcpyAsync(&l, m->d_scratch + kNParams, sizeof(float), cudaMemcpyDeviceToHost,
                               m->stream));
  LBM_MCUDA(m, cudaStreamSynchronize(m->stream));
  if (loss) *loss = l;
  return LBM_OK;
}

lbm_status lbm_mlp_train(lbm_mlp* m, const float* X, const float* Y, int n, const int* order,
                         int epochs, int batch, float lr, float* final_loss) {
  if (!m || !X || !Y || !order || n < 1 || epochs < 1 || batch < 1 || batch > kTrainThreads ||
      !(lr > 0.f))
    return mfail(m, LBM_E_INVAL, "need n, epochs >= 1, 1 <= batch <= 128, lr > 0");
  for (size_t k = 0; k < size_t(epochs) * n; ++k)
    if (order[k] < 0 || order[k] >= n) return mfail(m, LBM_E_INVAL, "order index out of range");
  MDeviceGuard guard(m->device);
  DevBuf dx, dy, dord;
  LBM_MCUDA(m, cudaMalloc(&dx.p, size_t(n) * kIn * sizeof(float)));
  LBM_MCUDA(m, cudaMalloc(&dy.p, size_t(n) * kOut * sizeof(float)));
  LBM_MCUDA(m, cudaMalloc(&dord.p, size_t(epochs) * n * sizeof(int)));
  LBM_MCUDA(m, cudaMemcpyAsync(dx.p, X, size_t(n) * kIn * sizeof(float), cudaMemcpyHostToDevice,
                               m->stream));
  LBM_MCUDA(m, cudaMemcpyAsync(dy.p, Y, size_t(n) * kOut * sizeof(float), cudaMemcpyHostToDevice,
                               m->stream));
  LBM_MCUDA(m, cudaMemcpyAsync(dord.p, order, size_t(epochs) * n * sizeof(int),
                               cudaMemcpyHostToDevice, m->stream));
  mlp_train_kernel<<<1, kTrainThreads, sizeof(TrainSmem), m->stream>>>(
      m->d_params, m->d_m, m->d_v, static_cast<float*>(dx.p), static_cast<float*>(dy.p), n,
      static_cast<int*>(dord.p), epochs, batch, lr, m->adam_t, 0, nullptr,
      m->d_scratch + kNParams);
  LBM_MCUDA(m, cudaGetLastError());
  count_launches(1);
  float l = 0.f;
  LBM_MCUDA(m, cudaMemcpyAsync(&l, m->d_scratch + kNParams, sizeof(float), cudaMemcpyDeviceToHost,
                               m->stream));
  LBM_MCUDA(m, cudaStreamSynchronize(m->stream));
  m->adam_t += epochs * ((n + batch - 1) / batch);
  if (final_loss) *final_loss = l;
  return LBM_OK;
}

lbm_status lbm_mlp_predict(lbm_mlp* m, const float* X, int n, float* Y) {
  if (!m || !X || !Y || n < 1) return mfail(m, LBM_E_INVAL, "bad argument");
  MDeviceGuard guard(m->device);
  DevBuf dx, dy;
  LBM_MCUDA(m, cudaMalloc(&dx.p, size_t(n) * kIn * sizeof(float)));
  LBM_MCUDA(m, cudaMalloc(&dy.p, size_t(n) * kOut * sizeof(float)));
  LBM_MCUDA(m, cudaMemcpyAsync(dx.p, X, size_t(n) * kIn * sizeof(float), cudaMemcpyHostToDevice,
                               m->stream));
  mlp_predict_kernel<<<(n + 255) / 256, 256, 0, m->stream>>>(
      m->d_params, static_cast<float*>(dx.p), n, static_cast<float*>(dy.p));
  LBM_MCUDA(m, cudaGetLastError());
  count_launches(1);
  LBM_MCUDA(m, cudaMemcpyAsync(Y, dy.p, size_t(n) * kOut * sizeof(float), cudaMemcpyDeviceToHost,
                               m->stream));
  LBM_MCUDA(m, cudaStreamSynchronize(m->stream));
  return LBM_OK;
}

}  // extern "C"
