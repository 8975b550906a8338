// C ABI of the pseudopotential D2Q9 library: context life cycle, argument
// validation, launch geometry, and host <-> device copies.  Every step of
// the method itself runs in the kernels of lbm_step_*.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_geometry.h"
#include "lbm_internal.h"

namespace lbm {

// One thread per cell: psi (Eqs. 8, 23) of the cell and its eight
// neighbours (periodic), the force of Eq. 3, and u = -F / (2 rho).
__global__ void rest_velocity_kernel(const double* __restrict__ rho, int nx, int ny,
                                     Phys<double> P, double* ux, double* uy, unsigned* status) {
  const size_t plane = size_t(nx) * ny;
  bool bad = false;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < plane;
       i += size_t(gridDim.x) * blockDim.x) {
    const int x = int(i % nx), y = int(i / nx);
    double sx = 0.0, sy = 0.0;
    for (int a = 1; a < kQ; ++a) {
      const int xn = (x + ex_of(a) + nx) % nx, yn = (y + ey_of(a) + ny) % ny;
      const double w = (ex_of(a) != 0 && ey_of(a) != 0) ? 1.0 / 12.0 : 1.0 / 3.0;
      const double pn = psi_of_rho(rho[size_t(yn) * nx + xn], P, bad);
      sx += w * pn * ex_of(a);
      sy += w * pn * ey_of(a);
    }
    const double r = rho[i];
    const double pc = psi_of_rho(r, P, bad);
    const double Fx = P.minus_G * pc * sx, Fy = P.minus_G * pc * sy;
    const bool ok = r > 0.0;
    ux[i] = ok ? -Fx / (2.0 * r) : 0.0;
    uy[i] = ok ? -Fy / (2.0 * r) : 0.0;
  }
  if (bad && status) atomicOr(status, kStatusInvalidInitFlag);
}

cudaError_t rest_velocity_launch(const double* rho, int nx, int ny, double RT, double a,
                                 double b, double G, double* ux, double* uy, unsigned* status,
                                 cudaStream_t s) {
  Phys<double> P{};
  P.RT = RT;
  P.a = a;
  P.b4 = b / 4.0;
  P.two_over_G = 2.0 / G;
  P.minus_G = -G;
  size_t blocks = (size_t(nx) * ny + 255) / 256;
  if (blocks > 65535u * 8u) blocks = 65535u * 8u;
  rest_velocity_kernel<<<int(blocks < 1 ? 1 : blocks), 256, 0, s>>>(rho, nx, ny, P, ux, uy,
                                                                    status);
  return cudaGetLastError();
}

static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned long long n) { g_launches += n; }

cudaError_t strip_launch_f32(int, int, const StripLaunch&, int, cudaStream_t);
cudaError_t strip_launch_f64(int, int, const StripLaunch&, int, cudaStream_t);
cudaError_t strip_launch_bf16(int, int, const StripLaunch&, int, cudaStream_t);
cudaError_t strip_launch_f16(int, int, const StripLaunch&, int, cudaStream_t);
cudaError_t strip_occupancy_f32(int, int, int*);
cudaError_t strip2_launch_f32(int, int, const StripLaunch&, int, cudaStream_t);
cudaError_t strip2_launch_f64(int, int, const StripLaunch&, int, cudaStream_t);
cudaError_t strip2_occupancy_f32(int, int, int*);
cudaError_t strip2_occupancy_f64(int, int, int*);
cudaError_t strip2_launch_bf16(int, int, const StripLaunch&, int, cudaStream_t);
cudaError_t strip2_launch_f16(int, int, const StripLaunch&, int, cudaStream_t);
cudaError_t strip2_occupancy_bf16(int, int, int*);
cudaError_t strip2_occupancy_f16(int, int, int*);
cudaError_t strip_tma_launch_f32(int, const StripLaunch&, int, cudaStream_t);
cudaError_t strip_tma_occupancy_f32(int, int*);
cudaError_t strip_occupancy_f64(int, int, int*);
cudaError_t strip_occupancy_bf16(int, int, int*);
cudaError_t strip_occupancy_f16(int, int, int*);
cudaError_t set_state_f32(void*, float*, int, int, int, size_t, const double*, const double*,
                          const double*, const double*, const EosCheck&, cudaStream_t);
cudaError_t set_state_f64(void*, float*, int, int, int, size_t, const double*, const double*,
                          const double*, const double*, const EosCheck&, cudaStream_t);
cudaError_t set_state_bf16(void*, float*, int, int, int, size_t, const double*, const double*,
                          const double*, const double*, const EosCheck&, cudaStream_t);
cudaError_t set_state_f16(void*, float*, int, int, int, size_t, const double*, const double*,
                          const double*, const double*, const EosCheck&, cudaStream_t);
cudaError_t get_state_f32(const void*, const float*, int, int, size_t, double*, cudaStream_t);
cudaError_t get_state_f64(const void*, const float*, int, int, size_t, double*, cudaStream_t);
cudaError_t get_state_bf16(const void*, const float*, int, int, size_t, double*, cudaStream_t);
cudaError_t get_state_f16(const void*, const float*, int, int, size_t, double*, cudaStream_t);
cudaError_t mass_f32(const void*, const float*, size_t, size_t, size_t, double*, int, double*,
                     cudaStream_t);
cudaError_t mass_f64(const void*, const float*, size_t, size_t, size_t, double*, int, double*,
                     cudaStream_t);
cudaError_t mass_bf16(const void*, const float*, size_t, size_t, size_t, double*, int, double*,
                     cudaStream_t);
cudaError_t mass_f16(const void*, const float*, size_t, size_t, size_t, double*, int, double*,
                     cudaStream_t);

cudaError_t strip_launch(int precision, int scheme, int mode, const StripLaunch& L, int grid,
                         cudaStream_t s) {
  switch (precision) {
    case kFP32: return strip_launch_f32(scheme, mode, L, grid, s);
    case kFP64: return strip_launch_f64(scheme, mode, L, grid, s);
    case kBF16Dev: return strip_launch_bf16(scheme, mode, L, grid, s);
    case kFP16Dev: return strip_launch_f16(scheme, mode, L, grid, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t strip_occupancy(int precision, int scheme, int mode, int* b) {
  switch (precision) {
    case kFP32: return strip_occupancy_f32(scheme, mode, b);
    case kFP64: return strip_occupancy_f64(scheme, mode, b);
    case kBF16Dev: return strip_occupancy_bf16(scheme, mode, b);
    case kFP16Dev: return strip_occupancy_f16(scheme, mode, b);
  }
  return cudaErrorInvalidValue;
}
cudaError_t strip2_launch(int precision, int scheme, int mode, const StripLaunch& L, int grid,
                          cudaStream_t s) {
  if (precision == kFP32) return strip2_launch_f32(scheme, mode, L, grid, s);
  if (precision == kFP64) return strip2_launch_f64(scheme, mode, L, grid, s);
  if (precision == kBF16Dev) return strip2_launch_bf16(scheme, mode, L, grid, s);
  if (precision == kFP16Dev) return strip2_launch_f16(scheme, mode, L, grid, s);
  return cudaErrorNotSupported;
}
cudaError_t strip2_occupancy(int precision, int scheme, int mode, int* b) {
  if (precision == kFP32) return strip2_occupancy_f32(scheme, mode, b);
  if (precision == kFP64) return strip2_occupancy_f64(scheme, mode, b);
  if (precision == kBF16Dev) return strip2_occupancy_bf16(scheme, mode, b);
  if (precision == kFP16Dev) return strip2_occupancy_f16(scheme, mode, b);
  return cudaErrorNotSupported;
}
cudaError_t strip_tma_launch(int precision, int scheme, const StripLaunch& L, int grid,
                             cudaStream_t s) {
  if (precision != kFP32) return cudaErrorNotSupported;
  return strip_tma_launch_f32(scheme, L, grid, s);
}
cudaError_t strip_tma_occupancy(int precision, int scheme, int* b) {
  if (precision != kFP32) return cudaErrorNotSupported;
  return strip_tma_occupancy_f32(scheme, b);
}
cudaError_t set_state_launch(int precision, void* dst, float* rd, int nx, int ny, int pitch,
                             size_t plane, const double* rho, const double* ux, const double* uy,
                             const double* f_in, const EosCheck& chk, cudaStream_t s) {
  switch (precision) {
    case kFP32: return set_state_f32(dst, rd, nx, ny, pitch, plane, rho, ux, uy, f_in, chk, s);
    case kFP64: return set_state_f64(dst, rd, nx, ny, pitch, plane, rho, ux, uy, f_in, chk, s);
    case kBF16Dev: return set_state_bf16(dst, rd, nx, ny, pitch, plane, rho, ux, uy, f_in, chk, s);
    case kFP16Dev: return set_state_f16(dst, rd, nx, ny, pitch, plane, rho, ux, uy, f_in, chk, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t get_state_launch(int precision, const void* src, const float* rs, int nx, int ny,
                             size_t plane, double* f_out, cudaStream_t s) {
  switch (precision) {
    case kFP32: return get_state_f32(src, rs, nx, ny, plane, f_out, s);
    case kFP64: return get_state_f64(src, rs, nx, ny, plane, f_out, s);
    case kBF16Dev: return get_state_bf16(src, rs, nx, ny, plane, f_out, s);
    case kFP16Dev: return get_state_f16(src, rs, nx, ny, plane, f_out, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t mass_launch(int precision, const void* src, const float* rs, size_t plane,
                        size_t first, size_t count, double* partial, int n_partial, double* out,
                        cudaStream_t s) {
  switch (precision) {
    case kFP32: return mass_f32(src, rs, plane, first, count, partial, n_partial, out, s);
    case kFP64: return mass_f64(src, rs, plane, first, count, partial, n_partial, out, s);
    case kBF16Dev: return mass_bf16(src, rs, plane, first, count, partial, n_partial, out, s);
    case kFP16Dev: return mass_f16(src, rs, plane, first, count, partial, n_partial, out, s);
  }
  return cudaErrorInvalidValue;
}

size_t storage_bytes(int precision) {
  switch (precision) {
    case kFP32: return 4;
    case kFP64: return 8;
    case kBF16Dev:
    case kFP16Dev: return 2;
  }
  return 0;
}

}  // namespace lbm

using namespace lbm;

static thread_local std::string g_create_error;

struct lbm_ctx {
  lbm_params p{};
  double T = 0.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* f[2] = {nullptr, nullptr};
  float* rho[2] = {nullptr, nullptr};
  int cur = 0;  // buffer holding the current state
  size_t plane = 0;
  unsigned* d_status = nullptr;
  unsigned* h_status = nullptr;  // pinned
  double* d_partial = nullptr;
  int n_partial = 0;
  double* d_scalar = nullptr;
  double* d_tmp = nullptr;  // 3 * plane doubles, allocated on first use
  double* d_pop = nullptr;  // 9 * plane doubles, allocated on first use
  bool initialized = false;
  int last_scheme = LBM_SCHEME_SC;
  int sm_count = 0;
  int band_rows_override = 0;
  double mrt[3] = {0.0, 0.0, 0.0};  // s_e, s_eps, s_q of the MRT scheme (<= 0: 1/tau)
  int variant = LBM_VARIANT_AUTO;
  // A band of a y-decomposed lattice keeps kGhostRows ghost rows below and
  // above its p.ny owned rows: ny_buf = p.ny + 2 kGhostRows rows in every
  // buffer, owned rows from row0 = kGhostRows.  A whole lattice has
  // ny_buf = p.ny and row0 = 0.
  bool band = false;
  int ny_buf = 0;
  int row0 = 0;
  cudaEvent_t packed = nullptr;  // overlapped band step: boundary rows packed
  // Step graphs of small lattices (queue_steps): one per buffer parity, with
  // the launch arguments of its first step.
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    StripLaunch L{};
    int scheme = -1, variant = -1, grid = 0;
  } graph[2];
  cudaStream_t cap_stream = nullptr;  // private stream the graphs are captured on
  // lbm_get_moments on large lattices: row chunks copied on copy_stream while
  // the next chunk is computed; obs_ev[k] marks chunk k computed, obs_ev[last]
  // the copies done.
  static constexpr int kObsChunks = 4;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t obs_ev[kObsChunks + 1] = {};
  std::string err;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

lbm_status fail(lbm_ctx* ctx, lbm_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

lbm_status cuda_fail(lbm_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, LBM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(ctx, call)                                  \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

EosCheck eos_check(lbm_ctx* c) {
  EosCheck k{};
  k.RT = c->p.R * c->T;
  k.a = c->p.a;
  k.b4 = c->p.b / 4.0;
  k.two_over_G = 2.0 / c->p.G;
  k.status = c->d_status;
  return k;
}

StripLaunch base_launch(lbm_ctx* c) {
  StripLaunch L{};
  L.nx = c->p.nx;
  L.ny = c->ny_buf;
  L.y_begin = c->row0;
  L.y_end = c->row0 + c->p.ny;
  L.out_row0 = c->row0;
  L.plane = c->plane;
  L.status = c->d_status;
  L.RT = c->p.R * c->T;
  L.a = c->p.a;
  L.b4 = c->p.b / 4.0;
  L.two_over_G = 2.0 / c->p.G;
  L.minus_G = -c->p.G;
  L.tau = 1.0;
  L.omega = 1.0;
  L.sigma_ups = 0.0;
  L.guo = 0.5;
  return L;
}

// Kernel variant of this context for a step (or an observe) launch
// (resolve_variant).
int pick_variant(const lbm_ctx* c, int mode) {
  return resolve_variant(c->variant, c->p.precision, c->p.nx, c->p.ny, c->sm_count,
                         mode == kStepMode);
}

// Warp-strip geometry of one wave (strip_geometry) over the resident warp
// slots of the variant's kernel.
lbm_status geometry(lbm_ctx* c, int scheme, int mode, StripLaunch& L, int& grid, int rows = -1) {
  int bps = 0;
  const int variant = pick_variant(c, mode);
  if (variant == LBM_VARIANT_STAGED)
    LBM_CUDA(c, strip_tma_occupancy(c->p.precision, scheme, &bps));
  else if (variant == LBM_VARIANT_PAIR)
    LBM_CUDA(c, strip2_occupancy(c->p.precision, scheme, mode, &bps));
  else
    LBM_CUDA(c, strip_occupancy(c->p.precision, scheme, mode, &bps));
  if (bps < 1) bps = 1;
  const int warps_per_cta = kStripCtaThreads / 32;
  const long long resident = (long long)c->sm_count * bps * warps_per_cta;
  const StripGeometry g = strip_geometry(c->p.nx, rows < 0 ? c->p.ny : rows, variant, resident,
                                         warps_per_cta, c->band_rows_override);
  L.n_strips = g.n_strips;
  L.band_rows = g.band_rows;
  L.n_bands = g.n_bands;
  grid = g.grid;
  return LBM_OK;
}

lbm_status ensure_tmp(lbm_ctx* c, double** buf, size_t count) {
  if (*buf) return LBM_OK;
  cudaError_t e = cudaMalloc(buf, count * sizeof(double));
  if (e != cudaSuccess) {
    *buf = nullptr;
    return fail(c, LBM_E_NOMEM, "cudaMalloc of a staging buffer failed");
  }
  return LBM_OK;
}

// Launch arguments of a step with relaxation time tau and sigma.
StripLaunch step_launch(lbm_ctx* c, double tau, double sigma) {
  StripLaunch L = base_launch(c);
  L.tau = tau;
  L.omega = 1.0 / tau;
  L.sigma_ups = sigma / (tau - 0.5);
  L.guo = 1.0 - 1.0 / (2.0 * tau);
  L.s_e = c->mrt[0] > 0.0 ? c->mrt[0] : 1.0 / tau;
  L.s_eps = c->mrt[1] > 0.0 ? c->mrt[1] : 1.0 / tau;
  L.s_q = c->mrt[2] > 0.0 ? c->mrt[2] : 1.0 / tau;
  return L;
}

// One step of buffer rows [r0, r1) from buffer s into buffer d (no flip).
lbm_status launch_rows(lbm_ctx* c, int scheme, StripLaunch L, int r0, int r1, int s, int d) {
  if (r1 <= r0) return LBM_OK;
  L.y_begin = r0;
  L.y_end = r1;
  L.src = c->f[s];
  L.dst = c->f[d];
  L.rho_src = c->rho[s];
  L.rho_dst = c->rho[d];
  int grid = 0;
  lbm_status st = geometry(c, scheme, kStepMode, L, grid, r1 - r0);
  if (st != LBM_OK) return st;
  const int variant = pick_variant(c, kStepMode);
  cudaError_t e =
      variant == LBM_VARIANT_STAGED
          ? strip_tma_launch(c->p.precision, scheme, L, grid, c->stream)
          : variant == LBM_VARIANT_PAIR
                ? strip2_launch(c->p.precision, scheme, kStepMode, L, grid, c->stream)
                : strip_launch(c->p.precision, scheme, kStepMode, L, grid, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
  count_launches(1);
  return LBM_OK;
}

// Steps per captured step graph (even: a replay leaves the state in the same
// buffer) and the lattice size up to which steps go through graphs.  With
// one launch per step a small lattice (64^2 to 256^2) takes a flat ~6.2 us
// per step however little it computes; a graph of the same kernels replays
// them with shorter gaps (~4 us per step there, a few per cent faster up to
// 2048^2).  From 4096^2 on the step's own time hides the gap.
constexpr int kGraphSteps = 16;
constexpr size_t kGraphMaxCells = size_t(2048) * 2048;

// One step kernel from buffer c->cur on `stream`, flipping c->cur.
cudaError_t launch_step(lbm_ctx* c, int scheme, StripLaunch& L, int grid, cudaStream_t stream) {
  const int s = c->cur, d = 1 - c->cur;
  L.src = c->f[s];
  L.dst = c->f[d];
  L.rho_src = c->rho[s];
  L.rho_dst = c->rho[d];
  const int variant = pick_variant(c, kStepMode);
  const cudaError_t e =
      variant == LBM_VARIANT_STAGED
          ? strip_tma_launch(c->p.precision, scheme, L, grid, stream)
          : variant == LBM_VARIANT_PAIR
                ? strip2_launch(c->p.precision, scheme, kStepMode, L, grid, stream)
                : strip_launch(c->p.precision, scheme, kStepMode, L, grid, stream);
  if (e == cudaSuccess) c->cur = d;
  return e;
}

// Every argument a step kernel reads, compared field by field.
bool same_launch(const StripLaunch& x, const StripLaunch& y) {
  return x.src == y.src && x.dst == y.dst && x.rho_src == y.rho_src && x.rho_dst == y.rho_dst &&
         x.out_rho == y.out_rho && x.out_vx == y.out_vx && x.out_vy == y.out_vy &&
         x.status == y.status && x.nx == y.nx && x.ny == y.ny && x.y_begin == y.y_begin &&
         x.y_end == y.y_end && x.out_row0 == y.out_row0 && x.n_strips == y.n_strips &&
         x.band_rows == y.band_rows && x.n_bands == y.n_bands && x.plane == y.plane &&
         x.RT == y.RT && x.a == y.a && x.b4 == y.b4 && x.two_over_G == y.two_over_G &&
         x.minus_G == y.minus_G && x.tau == y.tau && x.omega == y.omega &&
         x.sigma_ups == y.sigma_ups && x.guo == y.guo && x.s_e == y.s_e && x.s_eps == y.s_eps &&
         x.s_q == y.s_q;
}

// The cached graph of kGraphSteps steps from the current buffer, captured
// again when any kernel argument, the scheme, the kernel variant or the grid
// changed; nullptr when capture is unavailable (the caller then launches
// step by step).
cudaGraphExec_t step_graph(lbm_ctx* c, int scheme, StripLaunch L, int grid) {
  lbm_ctx::StepGraph& g = c->graph[c->cur];
  const int variant = pick_variant(c, kStepMode);
  L.src = c->f[c->cur];
  L.dst = c->f[1 - c->cur];
  L.rho_src = c->rho[c->cur];
  L.rho_dst = c->rho[1 - c->cur];
  if (g.exec && g.scheme == scheme && g.variant == variant && g.grid == grid &&
      same_launch(g.L, L))
    return g.exec;
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  if (!c->cap_stream &&
      cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
    return nullptr;
  }
  const StripLaunch first = L;  // the key: launch_step overwrites the buffers
  const int cur0 = c->cur;
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) ==
            cudaSuccess;
  for (int k = 0; ok && k < kGraphSteps; ++k)
    ok = launch_step(c, scheme, L, grid, c->cap_stream) == cudaSuccess;
  c->cur = cur0;  // capturing ran nothing
  const bool ended = cudaStreamEndCapture(c->cap_stream, &graph) == cudaSuccess;
  cudaGraphExec_t exec = nullptr;
  if (ok && ended && graph && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
    exec = nullptr;
  if (graph) cudaGraphDestroy(graph);
  if (!exec) {
    cudaGetLastError();
    return nullptr;
  }
  g.exec = exec;
  g.L = first;
  g.scheme = scheme;
  g.variant = variant;
  g.grid = grid;
  return exec;
}

lbm_status queue_steps(lbm_ctx* c, int n, int scheme, double tau, double sigma) {
  if (!c) return LBM_E_INVAL;
  if (n < 0) return fail(c, LBM_E_INVAL, "n must be >= 0");
  if (scheme < 0 || scheme > LBM_SCHEME_MRT) return fail(c, LBM_E_INVAL, "unknown scheme");
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(c, LBM_E_INVAL, "tau must be > 1/2");
  if (!std::isfinite(sigma)) return fail(c, LBM_E_INVAL, "sigma must be finite");
  if (!c->initialized) return fail(c, LBM_E_STATE, "state not initialised");
  if (c->band && n > 1)
    return fail(c, LBM_E_INVAL, "a band advances one step per call (exchange halos between)");
  if (n == 0) return LBM_OK;
  StripLaunch L = step_launch(c, tau, sigma);
  int grid = 0;
  lbm_status st = geometry(c, scheme, kStepMode, L, grid);
  if (st != LBM_OK) return st;
  int k = 0;
  // (not while the caller captures the context stream into a graph of its
  // own: the steps are then recorded one launch at a time)
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  if (!c->band && n >= kGraphSteps && size_t(c->p.nx) * c->p.ny <= kGraphMaxCells &&
      cudaStreamIsCapturing(c->stream, &capturing) != cudaSuccess) {
    cudaGetLastError();  // treated as capturing: plain launches
    capturing = cudaStreamCaptureStatusActive;
  }
  if (!c->band && n >= kGraphSteps && size_t(c->p.nx) * c->p.ny <= kGraphMaxCells &&
      capturing == cudaStreamCaptureStatusNone) {
    const cudaGraphExec_t g = step_graph(c, scheme, L, grid);
    if (g)
      for (; k + kGraphSteps <= n; k += kGraphSteps)
        LBM_CUDA(c, cudaGraphLaunch(g, c->stream));  // the state returns to c->cur
  }
  for (; k < n; ++k) {
    const cudaError_t e = launch_step(c, scheme, L, grid, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
  }
  count_launches((unsigned long long)n);
  c->last_scheme = scheme;
  return LBM_OK;
}

}  // namespace

namespace {

// f = f_eq(rho, u): u from the caller (ux, uy; NULL = 0) or, at_rest, the
// velocity of zero actual velocity computed on the device.
lbm_status init_state(lbm_ctx* c, const double* rho, const double* ux, const double* uy,
                      bool at_rest) {
  if (!c) return LBM_E_INVAL;
  if (!rho) return fail(c, LBM_E_INVAL, "rho is NULL");
  DeviceGuard guard(c->p.device);
  lbm_status st = ensure_tmp(c, &c->d_tmp, 3 * c->plane);
  if (st != LBM_OK) return st;
  const size_t bytes = c->plane * sizeof(double);
  // inputs are copied into device staging slices first (a DMA copy over the
  // CPU-GPU link runs faster than the kernel reading host memory in place)
  const double* in[3] = {rho, ux, uy};
  const double* dev[3] = {nullptr, nullptr, nullptr};
  for (int k = 0; k < 3; ++k) {
    if (!in[k]) continue;
    double* stage = c->d_tmp + k * c->plane;
    LBM_CUDA(c, cudaMemcpyAsync(stage, in[k], bytes, cudaMemcpyHostToDevice, c->stream));
    dev[k] = stage;
  }
  const double *d_rho = dev[0], *d_ux = dev[1], *d_uy = dev[2];
  LBM_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream));
  if (at_rest) {
    double* vu = c->d_tmp + c->plane;
    double* vv = c->d_tmp + 2 * c->plane;
    LBM_CUDA(c, rest_velocity_launch(d_rho, c->p.nx, c->ny_buf, c->p.R * c->T, c->p.a, c->p.b,
                                     c->p.G, vu, vv, c->d_status, c->stream));
    count_launches(1);
    d_ux = vu;
    d_uy = vv;
  }
  LBM_CUDA(c, set_state_launch(c->p.precision, c->f[c->cur], c->rho[c->cur], c->p.nx, c->ny_buf,
                               c->p.nx, c->plane, d_rho, d_ux, d_uy, nullptr, eos_check(c),
                               c->stream));
  count_launches(1);
  LBM_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(unsigned),
                              cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (*c->h_status & kStatusInvalidInitFlag) {
    c->initialized = false;
    cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
    cudaStreamSynchronize(c->stream);
    return fail(c, LBM_E_INVAL,
                "rho outside the domain of psi (rho <= 0, b rho/4 >= 1 or negative radicand)");
  }
  c->initialized = true;
  c->last_scheme = LBM_SCHEME_SC;
  return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_params(lbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->a = 1.0;
  p->b = 4.0;
  p->R = 1.0;
  p->G = -1.0;
  p->tc_mode = 0;
  p->precision = LBM_FP32;
  p->device = 0;
  p->cuda_stream = nullptr;
}

}  // extern "C"

namespace {

constexpr int kGhostRows = 2;  // the pull reaches one row, the psi stencil one more

lbm_status create_impl(const lbm_params* p, bool band, lbm_ctx** out) {
  g_create_error.clear();
  if (!p || !out) {
    g_create_error = "null argument";
    return LBM_E_INVAL;
  }
  *out = nullptr;
  const long long ny_buf = band ? (long long)p->ny + 2 * kGhostRows : p->ny;
  if (p->nx < 1 || p->ny < 1 || (long long)p->nx * ny_buf > 0x7fffffffLL) {
    g_create_error = "nx, ny must be >= 1 with nx * ny < 2^31";
    return LBM_E_INVAL;
  }
  if (band && p->ny < kGhostRows) {
    g_create_error = "a band must own at least 2 rows";
    return LBM_E_INVAL;
  }
  if (!(p->T_over_Tc > 0.0) || !(p->G < 0.0) || !(p->b > 0.0) || !(p->R > 0.0) ||
      !(p->a > 0.0)) {
    g_create_error = "need T_over_Tc > 0, G < 0, a, b, R > 0";
    return LBM_E_INVAL;
  }
  if (p->precision < LBM_FP32 || p->precision > LBM_FP16DEV) {
    g_create_error = "unknown precision";
    return LBM_E_INVAL;
  }
  double Tc = 0.0;
  if (p->tc_mode == 0) {
    double rc, pc;
    if (lbm_cs_critical_point(p->a, p->b, p->R, &rc, &Tc, &pc) != LBM_OK) {
      g_create_error = "critical point not found";
      return LBM_E_INVAL;
    }
  } else if (p->tc_mode == 1) {
    Tc = 0.094;
  } else {
    g_create_error = "tc_mode must be 0 or 1";
    return LBM_E_INVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) {
    g_create_error = "no such CUDA device";
    return LBM_E_CUDA;
  }
  DeviceGuard guard(p->device);
  lbm_ctx* c = new lbm_ctx();
  c->p = *p;
  c->T = p->T_over_Tc * Tc;
  c->band = band;
  c->ny_buf = int(ny_buf);
  c->row0 = band ? kGhostRows : 0;
  c->plane = (size_t)p->nx * ny_buf;
  auto bail = [&](lbm_status st, const char* msg) {
    g_create_error = msg;
    lbm_destroy(c);
    return st;
  };
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, p->device) !=
      cudaSuccess)
    return bail(LBM_E_CUDA, "cudaDeviceGetAttribute failed");
  if (p->cuda_stream) {
    c->stream = static_cast<cudaStream_t>(p->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(LBM_E_CUDA, "cudaStreamCreate failed");
    c->own_stream = true;
  }
  const size_t pop_bytes = 9 * c->plane * storage_bytes(p->precision);
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&c->f[i], pop_bytes) != cudaSuccess)
      return bail(LBM_E_NOMEM, "cudaMalloc of a population buffer failed");
    if (p->precision == LBM_BF16DEV || p->precision == LBM_FP16DEV) {
      if (cudaMalloc(&c->rho[i], c->plane * sizeof(float)) != cudaSuccess)
        return bail(LBM_E_NOMEM, "cudaMalloc of a density plane failed");
    }
  }
  c->n_partial = 2 * c->sm_count;
  if (cudaMalloc(&c->d_status, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&c->d_partial, c->n_partial * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_scalar, sizeof(double)) != cudaSuccess)
    return bail(LBM_E_NOMEM, "cudaMalloc of scratch failed");
  if (cudaMallocHost(&c->h_status, sizeof(unsigned)) != cudaSuccess)
    return bail(LBM_E_NOMEM, "cudaMallocHost failed");
  if (cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(LBM_E_CUDA, "status init failed");
  *out = c;
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_params* p, lbm_ctx** out) { return create_impl(p, false, out); }

lbm_status lbm_create_band(const lbm_params* p, lbm_ctx** out) {
  return create_impl(p, true, out);
}

lbm_status lbm_destroy(lbm_ctx* c) {
  if (!c) return LBM_OK;
  DeviceGuard guard(c->p.device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int i = 0; i < 2; ++i) {
    cudaFree(c->f[i]);
    cudaFree(c->rho[i]);
  }
  cudaFree(c->d_status);
  cudaFree(c->d_partial);
  cudaFree(c->d_scalar);
  cudaFree(c->d_tmp);
  cudaFree(c->d_pop);
  if (c->packed) cudaEventDestroy(c->packed);
  for (auto& g : c->graph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (cudaEvent_t e : c->obs_ev)
    if (e) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

lbm_status lbm_get_temperature(const lbm_ctx* c, double* T) {
  if (!c || !T) return LBM_E_INVAL;
  *T = c->T;
  return LBM_OK;
}

lbm_status lbm_init_density(lbm_ctx* c, const double* rho, const double* ux,
                            const double* uy) {
  return init_state(c, rho, ux, uy, false);
}

lbm_status lbm_init_density_at_rest(lbm_ctx* c, const double* rho) {
  return init_state(c, rho, nullptr, nullptr, true);
}

lbm_status lbm_step_async(lbm_ctx* c, int n, int scheme, double tau, double sigma) {
  if (!c) return LBM_E_INVAL;
  DeviceGuard guard(c->p.device);
  return queue_steps(c, n, scheme, tau, sigma);
}

lbm_status lbm_sync_status(lbm_ctx* c) {
  if (!c) return LBM_E_INVAL;
  DeviceGuard guard(c->p.device);
  LBM_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(unsigned),
                              cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (*c->h_status & kStatusTimeoutFlag) {
    cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
    cudaStreamSynchronize(c->stream);
    return fail(c, LBM_E_TIMEOUT, "a bounded wait for staged rows gave up");
  }
  if (*c->h_status & kStatusDivergedFlag)
    return fail(c, LBM_E_DIVERGED, "density left the domain of psi");
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int n, int scheme, double tau, double sigma) {
  lbm_status st = lbm_step_async(c, n, scheme, tau, sigma);
  if (st != LBM_OK) return st;
  return lbm_sync_status(c);
}

lbm_status lbm_get_moments(lbm_ctx* c, double* rho, double* vx, double* vy) {
  if (!c) return LBM_E_INVAL;
  if (!c->initialized) return fail(c, LBM_E_STATE, "state not initialised");
  DeviceGuard guard(c->p.device);
  lbm_status st = ensure_tmp(c, &c->d_tmp, 3 * c->plane);
  if (st != LBM_OK) return st;
  StripLaunch L = base_launch(c);
  L.src = c->f[c->cur];
  L.rho_src = c->rho[c->cur];
  // The kernel writes device staging slices, then one DMA copy per output
  // (on an 8192^2 lattice: 3 x 537 MB in ~8.4 ms from page-locked memory,
  // against 23 ms with the kernel writing page-locked host memory in place;
  // a NULL output is still written, to staging).  From 2048^2 cells on, the
  // rows go in kObsChunks chunks, each copied on copy_stream while the next
  // is computed, so only the first chunk's kernel is not hidden behind the
  // copies (the values do not depend on the chunking).
  double* out[3] = {rho, vx, vy};
  double* dev[3];
  for (int k = 0; k < 3; ++k) dev[k] = c->d_tmp + k * c->plane;
  L.out_rho = dev[0];
  L.out_vx = dev[1];
  L.out_vy = dev[2];
  const int mode = c->last_scheme == LBM_SCHEME_NOFORCE ? kObserveNoForceMode : kObserveMode;
  const int nx = c->p.nx, ny = c->p.ny;
  const bool any_out = rho || vx || vy;
  int chunks = size_t(nx) * ny >= size_t(2048) * 2048 && any_out ? lbm_ctx::kObsChunks : 1;
  if (chunks > 1 && !c->copy_stream) {
    bool ok = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; ok && k <= lbm_ctx::kObsChunks; ++k)
      ok = cudaEventCreateWithFlags(&c->obs_ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {  // one chunk on the context stream instead
      cudaGetLastError();
      for (cudaEvent_t& e : c->obs_ev)
        if (e) {
          cudaEventDestroy(e);
          e = nullptr;
        }
      if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
      c->copy_stream = nullptr;
    }
  }
  if (!c->copy_stream) chunks = 1;
  LBM_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream));
  const bool pair = pick_variant(c, mode) == LBM_VARIANT_PAIR;
  for (int k = 0; k < chunks; ++k) {
    const int r0 = int(size_t(ny) * k / chunks), r1 = int(size_t(ny) * (k + 1) / chunks);
    if (r1 == r0) continue;  // fewer rows than chunks
    L.y_begin = c->row0 + r0;
    L.y_end = c->row0 + r1;
    int grid = 0;
    st = geometry(c, LBM_SCHEME_SC, mode, L, grid, r1 - r0);
    if (st != LBM_OK) return st;
    LBM_CUDA(c, pair ? strip2_launch(c->p.precision, LBM_SCHEME_SC, mode, L, grid, c->stream)
                     : strip_launch(c->p.precision, LBM_SCHEME_SC, mode, L, grid, c->stream));
    count_launches(1);
    cudaStream_t cs = c->stream;
    if (chunks > 1) {
      LBM_CUDA(c, cudaEventRecord(c->obs_ev[k], c->stream));
      LBM_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->obs_ev[k], 0));
      cs = c->copy_stream;
    }
    const size_t off = size_t(r0) * nx, bytes = size_t(r1 - r0) * nx * sizeof(double);
    for (int a = 0; a < 3; ++a)
      if (out[a] && bytes)
        LBM_CUDA(c, cudaMemcpyAsync(out[a] + off, dev[a] + off, bytes, cudaMemcpyDeviceToHost,
                                    cs));
  }
  if (chunks > 1) {  // the context stream waits for the copies
    LBM_CUDA(c, cudaEventRecord(c->obs_ev[lbm_ctx::kObsChunks], c->copy_stream));
    LBM_CUDA(c, cudaStreamWaitEvent(c->stream, c->obs_ev[lbm_ctx::kObsChunks], 0));
  }
  return lbm_sync_status(c);
}

lbm_status lbm_get_mass(lbm_ctx* c, double* mass) {
  if (!c || !mass) return fail(c, LBM_E_INVAL, "null argument");
  if (!c->initialized) return fail(c, LBM_E_STATE, "state not initialised");
  DeviceGuard guard(c->p.device);
  LBM_CUDA(c, mass_launch(c->p.precision, c->f[c->cur], c->rho[c->cur], c->plane,
                          (size_t)c->row0 * c->p.nx, (size_t)c->p.ny * c->p.nx, c->d_partial,
                          c->n_partial, c->d_scalar, c->stream));
  count_launches(2);
  LBM_CUDA(c, cudaMemcpyAsync(mass, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* c, double* f) {
  if (!c || !f) return fail(c, LBM_E_INVAL, "null argument");
  if (!c->initialized) return fail(c, LBM_E_STATE, "state not initialised");
  DeviceGuard guard(c->p.device);
  lbm_status st = ensure_tmp(c, &c->d_pop, 9 * c->plane);
  if (st != LBM_OK) return st;
  LBM_CUDA(c, get_state_launch(c->p.precision, c->f[c->cur], c->rho[c->cur], c->p.nx,
                               c->ny_buf, c->plane, c->d_pop, c->stream));
  count_launches(1);
  // owned rows of every plane: [9][ny][nx]
  const size_t own = (size_t)c->p.nx * c->p.ny * sizeof(double);
  LBM_CUDA(c, cudaMemcpy2DAsync(f, own, c->d_pop + (size_t)c->row0 * c->p.nx,
                                c->plane * sizeof(double), own, 9, cudaMemcpyDeviceToHost,
                                c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* c, const double* f) {
  if (!c || !f) return fail(c, LBM_E_INVAL, "null argument");
  if (c->band) return fail(c, LBM_E_INVAL, "a band is set from a density (init) only");
  DeviceGuard guard(c->p.device);
  lbm_status st = ensure_tmp(c, &c->d_pop, 9 * c->plane);
  if (st != LBM_OK) return st;
  LBM_CUDA(c, cudaMemcpyAsync(c->d_pop, f, 9 * c->plane * sizeof(double),
                              cudaMemcpyHostToDevice, c->stream));
  LBM_CUDA(c, set_state_launch(c->p.precision, c->f[c->cur], c->rho[c->cur], c->p.nx,
                               c->ny_buf, c->p.nx, c->plane, nullptr, nullptr, nullptr, c->d_pop,
                               EosCheck{}, c->stream));
  count_launches(1);
  LBM_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->initialized = true;
  return LBM_OK;
}

lbm_status lbm_band_halo_bytes(const lbm_ctx* c, size_t* bytes) {
  if (!c || !bytes) return LBM_E_INVAL;
  if (!c->band) return LBM_E_STATE;
  const size_t row = (size_t)c->p.nx;
  *bytes = kGhostRows * row * (9 * storage_bytes(c->p.precision) + (c->rho[0] ? 4 : 0));
  return LBM_OK;
}

}  // extern "C"

namespace {

// Copy kGhostRows rows starting at buffer row `row` of the current state to
// (to_msg) or from a packed message: [9][kGhostRows][nx] populations, then,
// for deviation storage, [kGhostRows][nx] of the density plane.
lbm_status halo_copy(lbm_ctx* c, int row, void* msg, bool to_msg) {
  const size_t sb = storage_bytes(c->p.precision);
  const size_t width = kGhostRows * (size_t)c->p.nx * sb;  // bytes of one plane's rows
  char* buf = static_cast<char*>(c->f[c->cur]) + (size_t)row * c->p.nx * sb;
  char* m = static_cast<char*>(msg);
  const size_t pitch = c->plane * sb;
  if (to_msg)
    LBM_CUDA(c, cudaMemcpy2DAsync(m, width, buf, pitch, width, 9, cudaMemcpyDeviceToDevice,
                                  c->stream));
  else
    LBM_CUDA(c, cudaMemcpy2DAsync(buf, pitch, m, width, width, 9, cudaMemcpyDeviceToDevice,
                                  c->stream));
  if (c->rho[c->cur]) {
    float* r = c->rho[c->cur] + (size_t)row * c->p.nx;
    char* mr = m + 9 * width;
    const size_t rb = kGhostRows * (size_t)c->p.nx * sizeof(float);
    if (to_msg)
      LBM_CUDA(c, cudaMemcpyAsync(mr, r, rb, cudaMemcpyDeviceToDevice, c->stream));
    else
      LBM_CUDA(c, cudaMemcpyAsync(r, mr, rb, cudaMemcpyDeviceToDevice, c->stream));
  }
  return LBM_OK;
}

lbm_status halo_check(lbm_ctx* c, const void* a, const void* b) {
  if (!c) return LBM_E_INVAL;
  if (!a || !b) return fail(c, LBM_E_INVAL, "null halo buffer");
  if (!c->band) return fail(c, LBM_E_STATE, "not a band context");
  if (!c->initialized) return fail(c, LBM_E_STATE, "state not initialised");
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_band_halo_pack(lbm_ctx* c, void* d_lo, void* d_hi) {
  lbm_status st = halo_check(c, d_lo, d_hi);
  if (st != LBM_OK) return st;
  DeviceGuard guard(c->p.device);
  st = halo_copy(c, c->row0, d_lo, true);  // the two lowest owned rows
  if (st != LBM_OK) return st;
  return halo_copy(c, c->row0 + c->p.ny - kGhostRows, d_hi, true);  // the two highest
}

lbm_status lbm_band_halo_unpack(lbm_ctx* c, const void* d_below, const void* d_above) {
  lbm_status st = halo_check(c, d_below, d_above);
  if (st != LBM_OK) return st;
  DeviceGuard guard(c->p.device);
  st = halo_copy(c, 0, const_cast<void*>(d_below), false);
  if (st != LBM_OK) return st;
  return halo_copy(c, c->row0 + c->p.ny, const_cast<void*>(d_above), false);
}

lbm_status lbm_band_step_overlap(lbm_ctx* c, int scheme, double tau, double sigma, void* d_lo,
                                 void* d_hi, void* comm_stream) {
  lbm_status st = halo_check(c, d_lo, d_hi);
  if (st != LBM_OK) return st;
  if (scheme < 0 || scheme > LBM_SCHEME_MRT) return fail(c, LBM_E_INVAL, "unknown scheme");
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(c, LBM_E_INVAL, "tau must be > 1/2");
  if (!std::isfinite(sigma)) return fail(c, LBM_E_INVAL, "sigma must be finite");
  DeviceGuard guard(c->p.device);
  if (!c->packed)
    LBM_CUDA(c, cudaEventCreateWithFlags(&c->packed, cudaEventDisableTiming));
  const StripLaunch L = step_launch(c, tau, sigma);
  const int s = c->cur, d = 1 - c->cur;
  const int r0 = c->row0, n = c->p.ny, g = kGhostRows;
  // the rows the neighbours need first: the two lowest and two highest
  // owned rows (all of them when the band is too thin to have an interior)
  const bool thin = n < 2 * g + 1;
  st = launch_rows(c, scheme, L, r0, thin ? r0 + n : r0 + g, s, d);
  if (st == LBM_OK && !thin) st = launch_rows(c, scheme, L, r0 + n - g, r0 + n, s, d);
  if (st != LBM_OK) return st;
  c->cur = d;  // the packs read the new state
  st = halo_copy(c, r0, d_lo, true);
  if (st == LBM_OK) st = halo_copy(c, r0 + n - g, d_hi, true);
  if (st != LBM_OK) return st;
  LBM_CUDA(c, cudaEventRecord(c->packed, c->stream));
  if (comm_stream)
    LBM_CUDA(c, cudaStreamWaitEvent(static_cast<cudaStream_t>(comm_stream), c->packed, 0));
  // the interior rows, while the messages travel
  if (!thin) st = launch_rows(c, scheme, L, r0 + g, r0 + n - g, s, d);
  if (st != LBM_OK) return st;
  c->last_scheme = scheme;
  return LBM_OK;
}

unsigned long long lbm_kernel_launch_count(void) { return g_launches.load(); }

lbm_status lbm_set_kernel_variant(lbm_ctx* c, int variant) {
  if (!c) return LBM_E_INVAL;
  if (variant < LBM_VARIANT_AUTO || variant > LBM_VARIANT_PAIR)
    return fail(c, LBM_E_INVAL, "unknown kernel variant");
  c->variant = variant;
  return LBM_OK;
}

lbm_status lbm_set_mrt_rates(lbm_ctx* c, double s_e, double s_eps, double s_q) {
  if (!c) return LBM_E_INVAL;
  for (double s : {s_e, s_eps, s_q})
    if (!std::isfinite(s) || !(s < 2.0)) return fail(c, LBM_E_INVAL, "MRT rates must be < 2");
  c->mrt[0] = s_e;
  c->mrt[1] = s_eps;
  c->mrt[2] = s_q;
  return LBM_OK;
}

lbm_status lbm_set_band_rows(lbm_ctx* c, int band_rows) {
  if (!c) return LBM_E_INVAL;
  if (band_rows < 0) return fail(c, LBM_E_INVAL, "band_rows must be >= 0");
  c->band_rows_override = band_rows;
  return LBM_OK;
}

lbm_status lbm_get_launch_geometry(lbm_ctx* c, int scheme, int* n_strips, int* band_rows,
                                   int* n_bands, int* grid) {
  if (!c) return LBM_E_INVAL;
  if (scheme < 0 || scheme > LBM_SCHEME_MRT) return fail(c, LBM_E_INVAL, "unknown scheme");
  DeviceGuard guard(c->p.device);
  StripLaunch L = base_launch(c);
  int g = 0;
  lbm_status st = geometry(c, scheme, kStepMode, L, g);
  if (st != LBM_OK) return st;
  if (n_strips) *n_strips = L.n_strips;
  if (band_rows) *band_rows = L.band_rows;
  if (n_bands) *n_bands = L.n_bands;
  if (grid) *grid = g;
  return LBM_OK;
}

lbm_status lbm_get_kernel_variant(lbm_ctx* c, int* variant) {
  if (!c || !variant) return LBM_E_INVAL;
  *variant = pick_variant(c, kStepMode);
  return LBM_OK;
}

}  // extern "C"
