// Batched parameter sweeps: many independent FP32 lattices advanced together.
//
// Every instance runs the fused step body of the single-domain kernels
// (strip_run2, two columns per lane; strip_run, one column per lane, for
// nx = 1 or when asked for; both in lbm_kernels.cuh) on its own slice of one
// packed buffer pair.  An odd-nx instance on the two-column body has rows of
// nx + 3 elements whose columns nx .. nx + 2 copy columns 0 .. 2 (refreshed
// every step: column nx by the pair store of the lane holding the last
// column, the other two by the lanes holding columns 1 and 2), so pairs stay
// aligned and the last column meets its periodic neighbours.  Instances fall
// in two classes by body, each with kernels of its own (separate register
// budgets).  A window of `window` steps is one CUDA graph, in one of
// three launch modes:
//   work list   -- per step, one launch per class; warps take strip x band
//                  items of the class's active instances from a prefix table
//                  (balanced for any mix of sizes); the two class kernels are
//                  two branches of the graph;
//   persistent  -- one launch per window and class; each CTA owns whole
//                  instances (longest-processing-time assignment) and only
//                  __syncthreads() separates its steps, so no CTA ever waits
//                  for another.  Small active sets then stay in L2;
//   cooperative -- one cooperative launch per window (every CTA resident);
//                  each step, warps take the work-list items of both classes,
//                  then all CTAs meet at a bounded grid barrier.
// All give bit-identical results (the band height never changes a value),
// so the window-level autotuner can try configurations on live windows.
// After each window one CTA per active instance reduces, in FP64, the row
// means (coexistence densities, width, mass) and the largest density change
// since the previous window (convergence), and flags non-finite values.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>
#include <queue>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_batch_host.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

struct BatchInst {
  size_t off;              // element offset of plane 0 in each population buffer
  size_t coff;             // cell offset in the density snapshot
  int nx, ny, n_strips;     // strips of 64 columns (pair) or 32
  int pitch;               // row pitch of the population planes: nx, or nx + 3 for odd nx
                           // on the two-column body (columns nx .. nx + 2 copy columns 0 .. 2)
  int pair;                // two columns per lane (strip_run2): even nx, and odd nx >= 3
  int band_rows, n_bands;  // work-list geometry
  int pband_rows, pn_bands;  // persistent geometry
  int scheme;
  int row_off;             // offset in the row-mean scratch
  Phys<float> P;
};

struct BatchOut {
  float max_dev;  // max over cells of |drho| / max(tol, 8 eps rho)
  float max_abs;  // max |drho|
  double rho_g, rho_l, width, mass;
  int finite;
};

constexpr int kWorklistThreads = 128;
#ifndef LBM_BATCH_PAIR_MIN_BLOCKS
#define LBM_BATCH_PAIR_MIN_BLOCKS 4  // CTAs per SM of the two-column work list (128 registers)
#endif
#ifndef LBM_BATCH_ODD_MIN_BLOCKS
#define LBM_BATCH_ODD_MIN_BLOCKS 6  // CTAs per SM of the one-column work list (80 registers)
#endif
constexpr int kPersistentThreads = 256;
constexpr int kReduceCta = 256;

__device__ __forceinline__ StripArgs<StoreF32> inst_args(const BatchInst& I, const float* src,
                                                        float* dst, unsigned* status,
                                                        bool persistent) {
  StripArgs<StoreF32> A;
  A.src = src + I.off;
  A.dst = dst + I.off;
  A.rho_src = nullptr;
  A.rho_dst = nullptr;
  A.out_rho = A.out_vx = A.out_vy = nullptr;
  A.status = status;
  A.nx = I.nx;
  A.ny = I.ny;
  A.pitch = I.pitch;
  A.y_begin = 0;
  A.y_end = I.ny;
  A.out_row0 = 0;
  A.n_strips = I.n_strips;
  A.band_rows = persistent ? I.pband_rows : I.band_rows;
  A.n_bands = persistent ? I.pn_bands : I.n_bands;
  A.plane = size_t(I.pitch) * I.ny;
  A.P = I.P;
  return A;
}

template <bool kPair, int SCHEME, bool kCoherent>
__device__ __forceinline__ void run_scheme(const StripArgs<StoreF32>& A, int strip, int band,
                                           int lane) {
  if constexpr (kPair)
    strip_run2<StoreF32, SCHEME, kModeStep, kCoherent, true, false>(A, strip, band, lane);
  else
    strip_run<StoreF32, SCHEME, kModeStep, kCoherent>(A, strip, band, lane);
}

template <bool kPair, bool kCoherent>
__device__ __forceinline__ void run_item(const StripArgs<StoreF32>& A, int scheme, int strip,
                                         int band, int lane) {
  // two bodies: the forced schemes share one (scheme read from A.P at run
  // time); the force-free one never evaluates psi
  if (scheme == kNoForce)
    run_scheme<kPair, kNoForce, kCoherent>(A, strip, band, lane);
  else
    run_scheme<kPair, kAnyForced, kCoherent>(A, strip, band, lane);
}

// The active list holds the two-column (even nx) instances first:
// counts[0] of them, then the others up to counts[1] = all active.  Each
// class has its own kernel instantiation (kPair), so neither body's register
// allocation constrains the other's.
__device__ __forceinline__ void class_range(const int* counts, bool pair, int& a0, int& a1) {
  a0 = pair ? 0 : counts[0];
  a1 = pair ? counts[0] : counts[1];
}

// Work-list item `item` (an index into the prefix table's range [a0, a1)):
// find its instance, stage the instance's arguments in the warp's shared
// slot (the body reloads them there instead of holding registers, like
// kernel parameters in the constant bank) and advance its strip x band.
template <bool kPair>
__device__ __forceinline__ void worklist_item(const BatchInst* __restrict__ inst,
                                              const int* __restrict__ active,
                                              const int* __restrict__ prefix, int a0, int a1,
                                              int item, const float* src, float* dst,
                                              unsigned* inst_status,
                                              StripArgs<StoreF32>& args, int lane) {
  int lo = a0, hi = a1;  // prefix[lo] <= item < prefix[lo + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= item) lo = mid; else hi = mid;
  }
  const int i = active[lo];
  const BatchInst I = inst[i];
  const int local = item - prefix[lo];
  __syncwarp();
  if (lane == 0) args = inst_args(I, src, dst, inst_status + i, false);
  __syncwarp();
  run_item<kPair, false>(args, I.scheme, local % I.n_strips, local / I.n_strips, lane);
}

// One step of every active instance of one class; warp w takes items
// w, w + W, ... of the class's range of the prefix table.
template <bool kPair>
__global__ void __launch_bounds__(kWorklistThreads,
                                  kPair ? LBM_BATCH_PAIR_MIN_BLOCKS : LBM_BATCH_ODD_MIN_BLOCKS)
batch_worklist_kernel(const BatchInst* __restrict__ inst, const int* __restrict__ active,
                      const int* __restrict__ prefix, const int* __restrict__ counts,
                      const float* src, float* dst, unsigned* inst_status) {
  __shared__ StripArgs<StoreF32> args[kWorklistThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = gridDim.x * (kWorklistThreads / 32);
  int a0, a1;
  class_range(counts, kPair, a0, a1);
  const int end = prefix[a1];
  for (int item = prefix[a0] + ((blockIdx.x * kWorklistThreads + threadIdx.x) >> 5); item < end;
       item += nwarps)
    worklist_item<kPair>(inst, active, prefix, a0, a1, item, src, dst, inst_status, args[warp],
                         lane);
}

// The same step with the items handed out dynamically: a warp that finishes
// an item takes the next one from the step's counter (zeroed at the start of
// the window), so warps whose items were short take more of them and the
// step ends when the work does, not when the unluckiest warp's fixed share
// does.  The order in which items are taken does not change any result.
template <bool kPair>
__global__ void __launch_bounds__(kWorklistThreads,
                                  kPair ? LBM_BATCH_PAIR_MIN_BLOCKS : LBM_BATCH_ODD_MIN_BLOCKS)
batch_worklist_dyn_kernel(const BatchInst* __restrict__ inst, const int* __restrict__ active,
                          const int* __restrict__ prefix, const int* __restrict__ counts,
                          const float* src, float* dst, unsigned* inst_status, int* counter) {
  __shared__ StripArgs<StoreF32> args[kWorklistThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int a0, a1;
  class_range(counts, kPair, a0, a1);
  const int first = prefix[a0], end = prefix[a1];
  for (;;) {
    int k = 0;
    if (lane == 0) k = atomicAdd(counter, 1);
    const int item = first + __shfl_sync(0xffffffffu, k, 0);
    if (item >= end) break;  // warp-uniform
    worklist_item<kPair>(inst, active, prefix, a0, a1, item, src, dst, inst_status, args[warp],
                         lane);
  }
}

// One step of every active instance of one class on the balanced one-wave
// schedule (balanced_schedule): warp w runs items[begin[w] .. begin[w + 1]),
// each a row range of one strip, together an equal share of the class's rows.
template <bool kPair>
__global__ void __launch_bounds__(kWorklistThreads,
                                  kPair ? LBM_BATCH_PAIR_MIN_BLOCKS : LBM_BATCH_ODD_MIN_BLOCKS)
batch_balanced_kernel(const BatchInst* __restrict__ inst, const int4* __restrict__ items,
                      const int* __restrict__ begin, const float* src, float* dst,
                      unsigned* inst_status) {
  __shared__ StripArgs<StoreF32> args[kWorklistThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = (blockIdx.x * kWorklistThreads + threadIdx.x) >> 5;
  const int k1 = begin[w + 1];
  for (int k = begin[w]; k < k1; ++k) {
    const int4 it = items[k];  // instance, strip, first row, end row
    const BatchInst I = inst[it.x];
    __syncwarp();
    if (lane == 0) {
      StripArgs<StoreF32> A = inst_args(I, src, dst, inst_status + it.x, false);
      A.y_begin = it.z;
      A.y_end = it.w;
      A.band_rows = it.w - it.z;
      A.n_bands = 1;
      args[warp] = A;
    }
    __syncwarp();
    run_item<kPair, false>(args[warp], I.scheme, it.y, 0, lane);
  }
}

// Grid barrier of the cooperative window: sync[0] counts arrivals, sync[1] is
// the generation, sync[2] the error word.  Every CTA is resident (cooperative
// launch), so the barrier completes; the wait is still bounded, and a CTA
// that gives up sets kStatusTimeout in sync[2] and the caller returns.
constexpr long long kBarrierSpinLimit = 1ll << 22;  // ~0.3-1 s of 64-ns sleeps

__device__ __forceinline__ bool grid_barrier(unsigned* sync) {
  __shared__ int ok_s;
  __syncthreads();  // every warp of this CTA finished the step
  if (threadIdx.x == 0) {
    volatile unsigned* gen = sync + 1;
    const unsigned g = *gen;  // read before arriving: the last arrival bumps it
    __threadfence();          // this CTA's stores of the step are visible device-wide
    bool ok = true;
    if (atomicAdd(sync, 1u) + 1u == gridDim.x) {
      atomicExch(sync, 0u);   // reset before releasing anyone
      __threadfence();
      atomicAdd(sync + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g && ++it < kBarrierSpinLimit) __nanosleep(64);
      ok = it < kBarrierSpinLimit;
      if (!ok) atomicOr(sync + 2, kStatusTimeout);
    }
    __threadfence();
    ok_s = ok && *(volatile unsigned*)(sync + 2) == 0u;
  }
  __syncthreads();
  return ok_s != 0;
}

// Self-test of the grid barrier's bounded wait: CTA 0 leaves without
// arriving (the arrival nothing makes), the others wait, give up after the
// spin limit, flag kStatusTimeout in sync[2] and return.
__global__ void __launch_bounds__(32) barrier_selftest_kernel(unsigned* sync) {
  if (blockIdx.x == 0) return;  // block-uniform
  grid_barrier(sync);
}

// `steps` steps of every active instance in one cooperative launch: in each
// step warps take items of both classes from the prefix table (the item body
// is chosen per instance), then all CTAs meet at the grid barrier.  Loads
// bypass L1 because other CTAs of this launch wrote them.
__global__ void __launch_bounds__(kWorklistThreads, LBM_BATCH_PAIR_MIN_BLOCKS)
batch_coop_kernel(const BatchInst* __restrict__ inst, const int* __restrict__ active,
                  const int* __restrict__ prefix, const int* __restrict__ counts, int steps,
                  float* buf0, float* buf1, unsigned* inst_status, unsigned* sync) {
  __shared__ StripArgs<StoreF32> args[kWorklistThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = gridDim.x * (kWorklistThreads / 32);
  const int na = counts[1];
  const int total = prefix[na];
  for (int s = 0; s < steps; ++s) {
    const float* src = (s & 1) ? buf1 : buf0;
    float* dst = (s & 1) ? buf0 : buf1;
    for (int item = (blockIdx.x * kWorklistThreads + threadIdx.x) >> 5; item < total;
         item += nwarps) {
      int lo = 0, hi = na;  // prefix[lo] <= item < prefix[lo + 1]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= item) lo = mid; else hi = mid;
      }
      const int i = active[lo];
      const BatchInst I = inst[i];
      const int local = item - prefix[lo];
      __syncwarp();
      // work-list geometry (the prefix table counts its items); coherent loads
      if (lane == 0) args[warp] = inst_args(I, src, dst, inst_status + i, false);
      __syncwarp();
      if (I.pair)  // warp-uniform
        run_item<true, true>(args[warp], I.scheme, local % I.n_strips, local / I.n_strips,
                             lane);
      else
        run_item<false, true>(args[warp], I.scheme, local % I.n_strips, local / I.n_strips,
                              lane);
    }
    if (!grid_barrier(sync)) return;
  }
}

// `steps` steps of the instances of one class this CTA owns (cta_begin and
// cta_list of that class); buffers alternate, starting from buf0.  The loads
// bypass L1 because this kernel wrote them.
template <bool kPair>
__global__ void __launch_bounds__(kPersistentThreads, 2)
batch_persistent_kernel(const BatchInst* __restrict__ inst, const int* __restrict__ cta_begin,
                        const int* __restrict__ cta_list, int steps, float* buf0, float* buf1,
                        unsigned* inst_status) {
  __shared__ StripArgs<StoreF32> args;
  const int k0 = cta_begin[blockIdx.x], k1 = cta_begin[blockIdx.x + 1];
  if (k0 >= k1) return;  // block-uniform
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kPersistentThreads / 32;
  for (int s = 0; s < steps; ++s) {
    const float* src = (s & 1) ? buf1 : buf0;
    float* dst = (s & 1) ? buf0 : buf1;
    for (int k = k0; k < k1; ++k) {
      const int i = cta_list[k];
      const BatchInst I = inst[i];
      __syncthreads();  // every warp is done with the previous instance's args
      if (threadIdx.x == 0) args = inst_args(I, src, dst, inst_status + i, true);
      __syncthreads();
      const int items = I.n_strips * I.pn_bands;
      for (int item = warp; item < items; item += kWarps)
        run_item<kPair, true>(args, I.scheme, item % I.n_strips, item / I.n_strips, lane);
    }
    __syncthreads();  // step s of every owned instance is complete
  }
}

__device__ __forceinline__ float pulled_rho(const float* f, size_t plane, int nx, int ny,
                                            int pitch, int x, int y) {
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const size_t r0 = size_t(y) * pitch, rm = size_t(ym) * pitch, rp = size_t(yp) * pitch;
  float r = f[r0 + x];
  r += f[plane + r0 + xm];
  r += f[2 * plane + rm + x];
  r += f[3 * plane + r0 + xp];
  r += f[4 * plane + rp + x];
  r += f[5 * plane + rm + xm];
  r += f[6 * plane + rm + xp];
  r += f[7 * plane + rp + xp];
  r += f[8 * plane + rp + xm];
  return r;
}

// One CTA per active instance: convergence against the snapshot, then the
// FP64 row means, coexistence densities, width and mass.
__global__ void __launch_bounds__(kReduceCta)
batch_window_reduce(const BatchInst* __restrict__ inst, const int* __restrict__ active,
                    const int* __restrict__ n_active_p, const float* cur, float* snap,
                    double* rowmean, BatchOut* out, float tol) {
  const int k = blockIdx.x;
  if (k >= *n_active_p) return;
  const int i = active[k];
  const BatchInst I = inst[i];
  __shared__ unsigned s_maxdev, s_maxabs;
  __shared__ int s_finite;
  if (threadIdx.x == 0) {
    s_maxdev = 0u;
    s_maxabs = 0u;
    s_finite = 1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t plane = size_t(I.pitch) * I.ny;
  const float* f = cur + I.off;
  float maxdev = 0.f, maxabs = 0.f;
  bool finite = true;
  for (int y = warp; y < I.ny; y += kReduceCta / 32) {
    double rs = 0.0;
    for (int x = lane; x < I.nx; x += 32) {
      const float r = pulled_rho(f, plane, I.nx, I.ny, I.pitch, x, y);
      float* sp = snap + I.coff + size_t(y) * I.nx + x;
      const float d = fabsf(r - *sp);
      const float thr = fmaxf(tol, 8.f * 1.1920929e-7f * fabsf(r));
      maxdev = fmaxf(maxdev, d / thr);
      maxabs = fmaxf(maxabs, d);
      finite = finite && isfinite(r);
      *sp = r;
      rs += double(r);
    }
    for (int o = 16; o > 0; o >>= 1) rs += __shfl_down_sync(0xffffffffu, rs, o);
    if (lane == 0) rowmean[I.row_off + y] = rs / I.nx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    maxdev = fmaxf(maxdev, __shfl_down_sync(0xffffffffu, maxdev, o));
    maxabs = fmaxf(maxabs, __shfl_down_sync(0xffffffffu, maxabs, o));
  }
  finite = __all_sync(0xffffffffu, finite);
  if (lane == 0) {
    atomicMax(&s_maxdev, __float_as_uint(maxdev));  // non-negative floats order as uints
    atomicMax(&s_maxabs, __float_as_uint(maxabs));
    if (!finite) s_finite = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double* rm = rowmean + I.row_off;
    const int ny = I.ny;
    const int lo = ny >= 2 ? ny / 2 - 1 : 0, hi = ny / 2;
    const double rg = 0.5 * (rm[0] + rm[ny - 1]);
    const double rl = 0.5 * (rm[lo] + rm[hi]);
    double gmax = 0.0, mass = 0.0;
    for (int y = 0; y < ny; ++y) {
      const double g = 0.5 * fabs(rm[y + 1 < ny ? y + 1 : 0] - rm[y > 0 ? y - 1 : ny - 1]);
      gmax = fmax(gmax, g);
      mass += rm[y];
    }
    BatchOut o;
    o.max_dev = __uint_as_float(s_maxdev);
    o.max_abs = __uint_as_float(s_maxabs);
    o.rho_g = rg;
    o.rho_l = rl;
    o.width = gmax > 0.0 ? (rl - rg) / gmax : 0.0;
    o.mass = mass * I.nx;
    o.finite = s_finite && isfinite(mass);
    out[i] = o;
  }
}

// Eq. 36 flat interface at rest for every instance (blockIdx.y = instance).
// For the smooth profile (W > 0) "at rest" means zero actual velocity
// v = u + F/(2 rho) (Table I): with the x-invariant profile F = (0, F_y),
// F_y = -G psi(y) (psi(y+1) - psi(y-1)) / 2 (Eq. 3 summed over the three
// neighbours in each row), so the equilibrium is taken at
// u = (0, -F_y / (2 rho)); starting at u = 0 instead gives the interface a
// velocity F/(2 rho) and a long transient.  For the sharp step (W <= 0) the
// force at the discontinuity is not that of any relaxed profile, so u = 0.
// Stored so that the next pull reproduces f_a(x) = f_eq_a(rho(y), u(y)).
__global__ void batch_init_slab_kernel(const BatchInst* __restrict__ inst,
                                       const double* __restrict__ prof, float* buf0,
                                       float* snap, unsigned* inst_status) {
  const int i = blockIdx.y;
  const BatchInst I = inst[i];
  const double rg = prof[3 * i], rl = prof[3 * i + 1], W = prof[3 * i + 2];
  const size_t plane = size_t(I.pitch) * I.ny;  // the profile is x-invariant: copies too
  const int ny = I.ny;
  auto wrap = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };
  auto rho_at = [&](int y) {
    y = wrap(y);
    if (W > 0.0)
      return rg + 0.5 * (rl - rg) *
                      (tanh(2.0 * (y - ny / 4.0) / W) - tanh(2.0 * (y - 3.0 * ny / 4.0) / W));
    return (y >= ny / 4 && y < 3 * ny / 4) ? rl : rg;
  };
  bool bad = false;
  auto psi_at = [&](int y) { return double(psi_of_rho(float(rho_at(y)), I.P, bad)); };
  auto uy_at = [&](int y) {
    const double Fy = double(I.P.minus_G) * psi_at(y) * 0.5 * (psi_at(y + 1) - psi_at(y - 1));
    return -Fy / (2.0 * rho_at(y));
  };
  for (size_t c = blockIdx.x * size_t(blockDim.x) + threadIdx.x; c < plane;
       c += size_t(gridDim.x) * blockDim.x) {
    const int y = int(c / I.pitch), x = int(c % I.pitch);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const int ys = y + ey_of(a);
      const double r = rho_at(ys);
      const double u = (I.scheme == kNoForce || W <= 0.0) ? 0.0 : uy_at(ys);
      const double eu = ey_of(a) * u;
      buf0[I.off + a * plane + c] =
          float(double(w_of<float>(a)) * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * u * u));
    }
    if (x < I.nx) snap[I.coff + size_t(y) * I.nx + x] = float(rho_at(y));
  }
  if (bad) atomicOr(inst_status + i, kStatusInvalidInit);
}

__global__ void batch_density_kernel(const BatchInst* __restrict__ inst, int i, const float* cur,
                                     double* out) {
  const BatchInst I = inst[i];
  const size_t plane = size_t(I.pitch) * I.ny, cells = size_t(I.nx) * I.ny;
  for (size_t c = blockIdx.x * size_t(blockDim.x) + threadIdx.x; c < cells;
       c += size_t(gridDim.x) * blockDim.x)
    out[c] = double(
        pulled_rho(cur + I.off, plane, I.nx, I.ny, I.pitch, int(c % I.nx), int(c / I.nx)));
}

// Density and actual velocity v = u + F/(2 rho) (Table I) of instance i,
// by the observe body of the single-domain kernel (one column per lane,
// 8-row bands).
template <int MODE>
__global__ void __launch_bounds__(kWorklistThreads)
batch_observe_kernel(const BatchInst* __restrict__ inst, int i, const float* cur, double* rho,
                     double* vx, double* vy, unsigned* inst_status) {
  const BatchInst I = inst[i];
  StripArgs<StoreF32> A = inst_args(I, cur, nullptr, inst_status + i, false);
  A.out_rho = rho;
  A.out_vx = vx;
  A.out_vy = vy;
  A.n_strips = (I.nx + 31) / 32;
  A.band_rows = 8;
  A.n_bands = (I.ny + 7) / 8;
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * kWorklistThreads + threadIdx.x) >> 5;
  if (w >= A.n_strips * A.n_bands) return;  // warp-uniform
  strip_run<StoreF32, kSC, MODE, false>(A, w % A.n_strips, w / A.n_strips, lane);
}

__global__ void to_float_kernel(const double* in, float* out, size_t n) {
  for (size_t c = blockIdx.x * size_t(blockDim.x) + threadIdx.x; c < n;
       c += size_t(gridDim.x) * blockDim.x)
    out[c] = float(in[c]);
}

}  // namespace lbm

using namespace lbm;

struct lbm_batch {
  lbm_batch_params p{};
  int count = 0;
  std::vector<lbm_instance> inst;
  std::vector<BatchInst> desc;
  std::vector<double> T;  // absolute temperature of each instance
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float* buf[2] = {nullptr, nullptr};
  float* snap = nullptr;
  double* rowmean = nullptr;
  BatchInst* d_inst = nullptr;
  BatchOut* d_out = nullptr;
  unsigned* d_status = nullptr;  // per instance
  double* d_prof = nullptr;      // 3 per instance
  double* d_tmp = nullptr;       // staging for one instance's density
  int* d_counters = nullptr;     // dynamic work list: item counter per step and class
  size_t tmp_cells = 0;
  // device work tables and their pinned host staging
  int* d_active = nullptr;
  int* d_prefix = nullptr;
  int* d_n_active = nullptr;     // {active two-column instances, all active}
  int* d_cta_begin = nullptr;
  int* d_cta_list = nullptr;
  int4* d_bal_items = nullptr;   // balanced schedule: items of class 0, then class 1
  int* d_bal_begin = nullptr;    // per class: wl_grid * 4 + 1 warp offsets
  int4* h_bal_items = nullptr;
  int* h_bal_begin = nullptr;
  int bal_cap = 0;               // items per class table
  int* h_active = nullptr;
  int* h_prefix = nullptr;
  int* h_cta_begin = nullptr;
  int* h_cta_list = nullptr;
  BatchOut* h_out = nullptr;
  unsigned* h_status = nullptr;
  std::vector<lbm_result> res;
  std::vector<ConvState> conv;  // per-instance state of the convergence rule
  std::vector<char> fresh;   // (re)initialised since the last window
  std::vector<int> active;
  int sm_count = 0;
  int wl_grid[2] = {0, 0};  // resident CTAs of each class's work-list kernel
  int pers_grid_max = 0;
  int coop_grid = 0;             // resident CTAs of the cooperative kernel (0: unsupported)
  unsigned* d_sync = nullptr;    // grid barrier: arrivals, generation, error
  cudaStream_t side = nullptr;   // second branch of the window graph
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // window graphs by (mode, grid of the two-column kernel, grid of the
  // one-column kernel); a grid of 0 leaves that class's kernel out
  std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
  int class_items[2] = {0, 0};  // work-list items of the active instances per class
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool initialized = false;
  WindowTuner tuner;  // launch configuration of LBM_BATCH_AUTO
  lbm_batch_stats stats{};
  std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status st, const std::string& m) {
  if (b) b->err = m;
  return st;
}

#define LBM_BCUDA(b, call)                                                               \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bfail(b, LBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

struct BDeviceGuard {
  int prev = -1;
  explicit BDeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~BDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Warps of the larger class's resident work-list wave (balanced tables).
int warps_max(const lbm_batch* b) {
  return std::max(b->wl_grid[0], b->wl_grid[1]) * (kWorklistThreads / 32);
}

void set_geometry(BatchInst& d, int rows) {
  d.band_rows = std::max(1, std::min(rows, d.ny));
  d.n_bands = (d.ny + d.band_rows - 1) / d.band_rows;
  const int want = (kPersistentThreads / 32 + d.n_strips - 1) / d.n_strips;  // fill 8 warps
  const int pb = std::max(1, std::min(want, d.ny));
  d.pband_rows = (d.ny + pb - 1) / pb;
  d.pn_bands = (d.ny + d.pband_rows - 1) / d.pband_rows;
}

constexpr int kBalancedMinRows = 8;

// Rebuild the active list (two-column instances first), the work-list prefix
// and the persistent assignment of each class; for a balanced window also
// each class's one-wave schedule.
lbm_status upload_tables(lbm_batch* b, int mode) {
  const int na = int(b->active.size());
  std::vector<int> cls[2];  // [0] two columns per lane, [1] one
  for (int i : b->active) cls[b->desc[i].pair ? 0 : 1].push_back(i);
  int acc = 0, k = 0;
  b->h_prefix[0] = 0;
  for (int c = 0; c < 2; ++c)
    for (int i : cls[c]) {
      const BatchInst& d = b->desc[i];
      b->h_active[k] = i;
      acc += d.n_strips * d.n_bands;
      b->h_prefix[++k] = acc;
    }
  b->class_items[0] = b->h_prefix[cls[0].size()];
  b->class_items[1] = acc - b->class_items[0];
  // the class counts ride at the end of the prefix staging
  b->h_prefix[b->count + 1] = int(cls[0].size());
  b->h_prefix[b->count + 2] = na;
  const int span = b->pers_grid_max + 1;
  const auto inst_cells = [b](int i) { return size_t(b->desc[i].nx) * b->desc[i].ny; };
  int pos = 0;
  for (int c = 0; c < 2; ++c)
    lpt_assign(cls[c], inst_cells, b->pers_grid_max, b->h_cta_begin + c * span, b->h_cta_list,
               pos);
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_inst, b->desc.data(), b->count * sizeof(BatchInst),
                               cudaMemcpyHostToDevice, b->stream));
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_active, b->h_active, std::max(na, 1) * sizeof(int),
                               cudaMemcpyHostToDevice, b->stream));
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_prefix, b->h_prefix, (na + 1) * sizeof(int),
                               cudaMemcpyHostToDevice, b->stream));
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_n_active, b->h_prefix + b->count + 1, 2 * sizeof(int),
                               cudaMemcpyHostToDevice, b->stream));
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_cta_begin, b->h_cta_begin,
                               2 * span * sizeof(int), cudaMemcpyHostToDevice,
                               b->stream));
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_cta_list, b->h_cta_list, std::max(pos, 1) * sizeof(int),
                               cudaMemcpyHostToDevice, b->stream));
  if (mode == LBM_BATCH_BALANCED)
    for (int c = 0; c < 2; ++c) {
      std::vector<BalColumn> cols;
      for (int i : cls[c]) cols.push_back(BalColumn{i, b->desc[i].n_strips, b->desc[i].ny});
      const int warps = b->wl_grid[c] * (kWorklistThreads / 32);
      int4* items = b->h_bal_items + size_t(c) * b->bal_cap;
      int* begin = b->h_bal_begin + size_t(c) * (warps_max(b) + 1);
      const int n = balanced_schedule(cols, warps, kBalancedMinRows,
                                      reinterpret_cast<BalItem*>(items), begin);
      LBM_BCUDA(b, cudaMemcpyAsync(b->d_bal_items + size_t(c) * b->bal_cap, items,
                                   std::max(n, 1) * sizeof(int4), cudaMemcpyHostToDevice,
                                   b->stream));
      LBM_BCUDA(b, cudaMemcpyAsync(b->d_bal_begin + size_t(c) * (warps_max(b) + 1), begin,
                                   (warps + 1) * sizeof(int), cudaMemcpyHostToDevice,
                                   b->stream));
    }
  return LBM_OK;
}

// Grid of a class kernel for the current active set (worklist_grid for the
// work list); 0 when the class has no active instance.
int class_grid(const lbm_batch* b, int mode, int cls) {
  if (b->class_items[cls] == 0) return 0;
  if (mode == LBM_BATCH_PERSISTENT) return b->pers_grid_max;
  if (mode == LBM_BATCH_BALANCED) return b->wl_grid[cls];
  return worklist_grid(b->class_items[cls], kWorklistThreads / 32, b->wl_grid[cls]);
}

// One window as a CUDA graph, captured once per (mode, class grids) and
// cached: the kernels read the active set and geometry from device memory,
// so the graph stays valid as instances leave.
lbm_status window_graph(lbm_batch* b, int mode, cudaGraphExec_t* out) {
  const bool coop = mode == LBM_BATCH_COOPERATIVE;
  const int g0 = coop ? b->coop_grid : class_grid(b, mode, 0);
  const int g1 = coop ? 0 : class_grid(b, mode, 1);
  const auto key = std::make_tuple(mode, g0, g1);
  const auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    *out = it->second;
    return LBM_OK;
  }
  cudaGraph_t g = nullptr;
  LBM_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  const int W = b->p.window;
  const int span = b->pers_grid_max + 1;
  // with both classes active they run as two branches of the graph, joined
  // after each step (work list) or before the reduction (persistent).  (Run
  // one after the other, each over the whole GPU, single-class batches gained
  // 6-13 % but the mixed 128-slab sweep lost 6 %.)
  const bool both = g0 > 0 && g1 > 0;
  cudaStream_t s1 = both ? b->side : b->stream;
  auto fork = [&]() {
    if (!both) return;
    cudaEventRecord(b->ev_fork, b->stream);
    cudaStreamWaitEvent(b->side, b->ev_fork, 0);
  };
  auto join = [&]() {
    if (!both) return;
    cudaEventRecord(b->ev_join, b->side);
    cudaStreamWaitEvent(b->stream, b->ev_join, 0);
  };
  if (coop) {
    // one cooperative launch for the whole window (barrier state reset first)
    cudaMemsetAsync(b->d_sync, 0, 3 * sizeof(unsigned), b->stream);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(b->coop_grid));
    cfg.blockDim = dim3(kWorklistThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(
        &cfg, batch_coop_kernel, static_cast<const BatchInst*>(b->d_inst),
        static_cast<const int*>(b->d_active), static_cast<const int*>(b->d_prefix),
        static_cast<const int*>(b->d_n_active), W, b->buf[0], b->buf[1], b->d_status,
        b->d_sync);
    if (le != cudaSuccess) {
      cudaGraph_t dead = nullptr;
      cudaStreamEndCapture(b->stream, &dead);
      if (dead) cudaGraphDestroy(dead);
      cudaGetLastError();
      return bfail(b, LBM_E_CUDA, std::string("cooperative launch: ") + cudaGetErrorString(le));
    }
  } else if (mode == LBM_BATCH_WORKLIST) {
    for (int s = 0; s < W; ++s) {
      fork();
      if (g0 > 0)
        batch_worklist_kernel<true><<<g0, kWorklistThreads, 0, b->stream>>>(
            b->d_inst, b->d_active, b->d_prefix, b->d_n_active, b->buf[s & 1],
            b->buf[(s + 1) & 1], b->d_status);
      if (g1 > 0)
        batch_worklist_kernel<false><<<g1, kWorklistThreads, 0, s1>>>(
            b->d_inst, b->d_active, b->d_prefix, b->d_n_active, b->buf[s & 1],
            b->buf[(s + 1) & 1], b->d_status);
      join();
    }
  } else if (mode == LBM_BATCH_WORKLIST_DYNAMIC) {
    // one item counter per step and class, zeroed once per window
    cudaMemsetAsync(b->d_counters, 0, 2 * size_t(W) * sizeof(int), b->stream);
    for (int s = 0; s < W; ++s) {
      fork();
      if (g0 > 0)
        batch_worklist_dyn_kernel<true><<<g0, kWorklistThreads, 0, b->stream>>>(
            b->d_inst, b->d_active, b->d_prefix, b->d_n_active, b->buf[s & 1],
            b->buf[(s + 1) & 1], b->d_status, b->d_counters + s);
      if (g1 > 0)
        batch_worklist_dyn_kernel<false><<<g1, kWorklistThreads, 0, s1>>>(
            b->d_inst, b->d_active, b->d_prefix, b->d_n_active, b->buf[s & 1],
            b->buf[(s + 1) & 1], b->d_status, b->d_counters + W + s);
      join();
    }
  } else if (mode == LBM_BATCH_BALANCED) {
    const int bspan = warps_max(b) + 1;
    for (int s = 0; s < W; ++s) {
      fork();
      if (g0 > 0)
        batch_balanced_kernel<true><<<g0, kWorklistThreads, 0, b->stream>>>(
            b->d_inst, b->d_bal_items, b->d_bal_begin, b->buf[s & 1], b->buf[(s + 1) & 1],
            b->d_status);
      if (g1 > 0)
        batch_balanced_kernel<false><<<g1, kWorklistThreads, 0, s1>>>(
            b->d_inst, b->d_bal_items + b->bal_cap, b->d_bal_begin + bspan, b->buf[s & 1],
            b->buf[(s + 1) & 1], b->d_status);
      join();
    }
  } else {
    fork();
    if (g0 > 0)
      batch_persistent_kernel<true><<<g0, kPersistentThreads, 0, b->stream>>>(
          b->d_inst, b->d_cta_begin, b->d_cta_list, W, b->buf[0], b->buf[1], b->d_status);
    if (g1 > 0)
      batch_persistent_kernel<false><<<g1, kPersistentThreads, 0, s1>>>(
          b->d_inst, b->d_cta_begin + span, b->d_cta_list, W, b->buf[0], b->buf[1],
          b->d_status);
    join();
  }
  batch_window_reduce<<<b->count, kReduceCta, 0, b->stream>>>(
      b->d_inst, b->d_active, b->d_n_active + 1, b->buf[0], b->snap, b->rowmean, b->d_out,
      float(b->p.tol));
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, LBM_E_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, LBM_E_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  }
  b->graphs[key] = exec;
  *out = exec;
  return LBM_OK;
}

size_t active_cells(const lbm_batch* b) {
  size_t c = 0;
  for (int i : b->active) c += size_t(b->desc[i].nx) * b->desc[i].ny;
  return c;
}

size_t max_active_cells(const lbm_batch* b) {
  size_t m = 0;
  for (int i : b->active) m = std::max(m, size_t(b->desc[i].nx) * b->desc[i].ny);
  return m;
}

// Launch configuration of the next window: the requested one, or the
// autotuner's (WindowTuner) under LBM_BATCH_AUTO.
void choose_config(lbm_batch* b, int& mode, int& rows) {
  if (b->p.mode != LBM_BATCH_AUTO) {
    mode = b->p.mode;
    rows = b->p.rows_per_item > 0 ? b->p.rows_per_item : 32;
    return;
  }
  const size_t cells = active_cells(b);
  const auto eligible = [&](size_t k) {
    const auto& c = b->tuner.candidates[k];
    if (b->p.rows_per_item > 0 &&
        (((c.first == LBM_BATCH_WORKLIST || c.first == LBM_BATCH_WORKLIST_DYNAMIC) &&
          c.second != b->p.rows_per_item) ||
         c.first == LBM_BATCH_BALANCED))
      return false;
    // a persistent window puts each instance on one SM: only worth trying
    // when the active populations are within a few times the L2 size and no
    // single instance is large
    if (c.first == LBM_BATCH_PERSISTENT &&
        (cells * 72 > size_t(512) << 20 || max_active_cells(b) > 65536))
      return false;
    return !(c.first == LBM_BATCH_COOPERATIVE && b->coop_grid == 0);
  };
  const auto choice = b->tuner.choose(cells, eligible);
  mode = choice.first;
  rows = choice.second;
}

}  // namespace

extern "C" {

void lbm_batch_default_params(lbm_batch_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->a = 1.0;
  p->b = 4.0;
  p->R = 1.0;
  p->G = -1.0;
  p->window = 1000;
  p->tol = 1e-9;
  p->max_steps = 200000;
  p->mode = LBM_BATCH_AUTO;
  p->conv_rel = 8.0 * 1.1920928955078125e-7;  // 8 ulp of FP32
  p->trend_tol = 1e-4;
}

lbm_status lbm_batch_create(const lbm_batch_params* p, const lbm_instance* in, int count,
                            lbm_batch** out) {
  if (!p || !in || !out || count < 1) return LBM_E_INVAL;
  *out = nullptr;
  if (p->window < 2 || p->window % 2 || p->max_steps < 1 || !(p->tol >= 0) ||
      p->mode < LBM_BATCH_AUTO || p->mode > LBM_BATCH_BALANCED || p->rows_per_item < 0 ||
      p->conv < LBM_CONV_COEX || p->conv > LBM_CONV_TREND || !(p->conv_rel >= 0.0) ||
      !(p->trend_tol >= 0.0) ||
      !(p->variant == LBM_VARIANT_AUTO || p->variant == LBM_VARIANT_PAIR ||
        p->variant == LBM_VARIANT_REGISTER) ||
      !(p->G < 0) || !(p->a > 0) || !(p->b > 0) || !(p->R > 0) || p->tc_mode < 0 ||
      p->tc_mode > 1)
    return LBM_E_INVAL;
  double Tc = 0.094, rc, pc;
  if (p->tc_mode == 0 && lbm_cs_critical_point(p->a, p->b, p->R, &rc, &Tc, &pc) != LBM_OK)
    return LBM_E_INVAL;
  for (int i = 0; i < count; ++i) {
    const lbm_instance& s = in[i];
    if (s.nx < 1 || s.ny < 1 || (long long)s.nx * s.ny > (1LL << 28) || !(s.T_over_Tc > 0) ||
        !(s.tau > 0.5) || !std::isfinite(s.tau) || !std::isfinite(s.sigma) || s.scheme < 0 ||
        s.scheme > LBM_SCHEME_LADD)
      return LBM_E_INVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev)
    return LBM_E_CUDA;
  BDeviceGuard guard(p->device);
  lbm_batch* b = new lbm_batch();
  b->p = *p;
  b->count = count;
  b->inst.assign(in, in + count);
  b->desc.resize(count);
  size_t off = 0, coff = 0;
  int roff = 0, max_cells = 0;
  for (int i = 0; i < count; ++i) {
    BatchInst& d = b->desc[i];
    const lbm_instance& s = in[i];
    d.off = off;
    d.coff = coff;
    d.nx = s.nx;
    d.ny = s.ny;
    d.pair = (s.nx % 2 == 0 || s.nx >= 3) && p->variant != LBM_VARIANT_REGISTER;
    d.pitch = d.pair && s.nx % 2 ? s.nx + 3 : s.nx;
    d.n_strips = d.pair ? (s.nx + 63) / 64 : (s.nx + 31) / 32;
    d.scheme = s.scheme;
    d.row_off = roff;
    const double T = s.T_over_Tc * Tc;
    b->T.push_back(T);
    d.P.RT = float(p->R * T);
    d.P.a = float(p->a);
    d.P.b4 = float(p->b / 4.0);
    d.P.two_over_G = float(2.0 / p->G);
    d.P.minus_G = float(-p->G);
    d.P.tau = float(s.tau);
    d.P.omega = float(1.0 / s.tau);
    d.P.sigma_ups = float(s.sigma / (s.tau - 0.5));
    d.P.guo = float(1.0 - 1.0 / (2.0 * s.tau));
    d.P.scheme = s.scheme;
    d.P.s_e = d.P.s_eps = d.P.s_q = d.P.omega;  // unused: the batch has no MRT scheme
    set_geometry(d, 32);
    const size_t cells = size_t(s.nx) * s.ny;
    off += (9 * size_t(d.pitch) * s.ny + 31) / 32 * 32;
    coff += cells;
    roff += s.ny;
    max_cells = std::max<int>(max_cells, int(cells));
  }
  b->tmp_cells = max_cells;
  b->res.assign(count, lbm_result{});
  b->conv.assign(count, ConvState{});
  b->fresh.assign(count, 1);
  auto bail = [&](lbm_status st, const char* m) {
    lbm_batch_destroy(b);
    (void)m;
    return st;
  };
  if (cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, p->device) !=
      cudaSuccess)
    return bail(LBM_E_CUDA, "attribute");
  if (p->cuda_stream) {
    b->stream = static_cast<cudaStream_t>(p->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(LBM_E_CUDA, "stream");
    b->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess)
    return bail(LBM_E_CUDA, "stream");
  int occ_wl[2] = {0, 0}, occ_p[2] = {0, 0};
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_wl[0], batch_worklist_kernel<true>,
                                                    kWorklistThreads, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_wl[1], batch_worklist_kernel<false>,
                                                    kWorklistThreads, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p[0], batch_persistent_kernel<true>,
                                                    kPersistentThreads, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p[1], batch_persistent_kernel<false>,
                                                    kPersistentThreads, 0) != cudaSuccess)
    return bail(LBM_E_CUDA, "occupancy");
  for (int c = 0; c < 2; ++c) b->wl_grid[c] = std::max(1, occ_wl[c]) * b->sm_count;
  b->pers_grid_max = std::max(1, std::min(occ_p[0], occ_p[1])) * b->sm_count;
  bool ok = true;
  ok &= cudaMalloc(&b->buf[0], off * sizeof(float)) == cudaSuccess;
  ok &= cudaMalloc(&b->buf[1], off * sizeof(float)) == cudaSuccess;
  ok &= cudaMalloc(&b->snap, coff * sizeof(float)) == cudaSuccess;
  ok &= cudaMalloc(&b->rowmean, roff * sizeof(double)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_inst, count * sizeof(BatchInst)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_out, count * sizeof(BatchOut)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_status, count * sizeof(unsigned)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_prof, 3 * count * sizeof(double)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_tmp, 3 * b->tmp_cells * sizeof(double)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_counters, 2 * size_t(p->window) * sizeof(int)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_active, count * sizeof(int)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_prefix, (count + 1) * sizeof(int)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_n_active, 2 * sizeof(int)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_cta_begin, 2 * (b->pers_grid_max + 1) * sizeof(int)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_cta_list, count * sizeof(int)) == cudaSuccess;
  ok &= cudaMalloc(&b->d_sync, 3 * sizeof(unsigned)) == cudaSuccess;
  {
    // balanced schedule: at most one item per warp plus one per strip boundary
    long long strips = 0;
    for (const BatchInst& d : b->desc) strips += d.n_strips;
    b->bal_cap = int(warps_max(b) + strips + 1);
    ok &= cudaMalloc(&b->d_bal_items, 2 * size_t(b->bal_cap) * sizeof(int4)) == cudaSuccess;
    ok &= cudaMalloc(&b->d_bal_begin, 2 * size_t(warps_max(b) + 1) * sizeof(int)) ==
          cudaSuccess;
  }
  if (!ok) return bail(LBM_E_NOMEM, "cudaMalloc");
  ok &= cudaMallocHost(&b->h_active, count * sizeof(int)) == cudaSuccess;
  ok &= cudaMallocHost(&b->h_prefix, (count + 3) * sizeof(int)) == cudaSuccess;
  ok &= cudaMallocHost(&b->h_cta_begin, 2 * (b->pers_grid_max + 1) * sizeof(int)) ==
        cudaSuccess;
  ok &= cudaMallocHost(&b->h_cta_list, count * sizeof(int)) == cudaSuccess;
  ok &= cudaMallocHost(&b->h_out, count * sizeof(BatchOut)) == cudaSuccess;
  ok &= cudaMallocHost(&b->h_status, count * sizeof(unsigned)) == cudaSuccess;
  ok &= cudaMallocHost(&b->h_bal_items, 2 * size_t(b->bal_cap) * sizeof(int4)) == cudaSuccess;
  ok &= cudaMallocHost(&b->h_bal_begin, 2 * size_t(warps_max(b) + 1) * sizeof(int)) ==
        cudaSuccess;
  if (!ok) return bail(LBM_E_NOMEM, "cudaMallocHost");
  if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return bail(LBM_E_CUDA, "event");
  if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)
    return bail(LBM_E_CUDA, "event");
  if (cudaMemsetAsync(b->d_status, 0, count * sizeof(unsigned), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->buf[0], 0, off * sizeof(float), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->buf[1], 0, off * sizeof(float), b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return bail(LBM_E_CUDA, "memset");
  for (int rows : {8, 16, 32, 64, 128}) b->tuner.add(LBM_BATCH_WORKLIST, rows);
  for (int rows : {8, 16, 32, 64}) b->tuner.add(LBM_BATCH_WORKLIST_DYNAMIC, rows);
  b->tuner.add(LBM_BATCH_BALANCED, 0);
  b->tuner.add(LBM_BATCH_PERSISTENT, 0);
  {
    // cooperative windows: every CTA resident, one launch per window
    int coop = 0, occ = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, p->device) == cudaSuccess &&
        coop &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_coop_kernel,
                                                      kWorklistThreads, 0) == cudaSuccess &&
        occ > 0)
      b->coop_grid = occ * b->sm_count;
    cudaGetLastError();
    if (b->coop_grid > 0)
      for (int rows : {16, 32, 64}) b->tuner.add(LBM_BATCH_COOPERATIVE, rows);
  }
  for (int i = 0; i < count; ++i) b->active.push_back(i);
  b->stats.n_active = count;
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  BDeviceGuard guard(b->p.device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  cudaFree(b->buf[0]);
  cudaFree(b->buf[1]);
  cudaFree(b->snap);
  cudaFree(b->rowmean);
  cudaFree(b->d_inst);
  cudaFree(b->d_out);
  cudaFree(b->d_status);
  cudaFree(b->d_prof);
  cudaFree(b->d_tmp);
  cudaFree(b->d_counters);
  cudaFree(b->d_active);
  cudaFree(b->d_prefix);
  cudaFree(b->d_n_active);
  cudaFree(b->d_cta_begin);
  cudaFree(b->d_cta_list);
  cudaFree(b->d_sync);
  cudaFree(b->d_bal_items);
  cudaFree(b->d_bal_begin);
  if (b->h_bal_items) cudaFreeHost(b->h_bal_items);
  if (b->h_bal_begin) cudaFreeHost(b->h_bal_begin);
  if (b->h_active) cudaFreeHost(b->h_active);
  if (b->h_prefix) cudaFreeHost(b->h_prefix);
  if (b->h_cta_begin) cudaFreeHost(b->h_cta_begin);
  if (b->h_cta_list) cudaFreeHost(b->h_cta_list);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->h_status) cudaFreeHost(b->h_status);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"

namespace {

// Instance i from f_eq(rho, u): u = 0, or at_rest the velocity of zero
// actual velocity computed on the device (rest_velocity_launch).
lbm_status batch_init_state(lbm_batch* b, int i, const double* rho, bool at_rest) {
  if (!b || !rho || i < 0 || i >= b->count) return bfail(b, LBM_E_INVAL, "bad argument");
  BDeviceGuard guard(b->p.device);
  const BatchInst& d = b->desc[i];
  const size_t cells = size_t(d.nx) * d.ny;
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_tmp, rho, cells * sizeof(double), cudaMemcpyHostToDevice,
                               b->stream));
  LBM_BCUDA(b, cudaMemsetAsync(b->d_status + i, 0, sizeof(unsigned), b->stream));
  EosCheck chk{};
  chk.RT = double(d.P.RT);
  chk.a = double(d.P.a);
  chk.b4 = double(d.P.b4);
  chk.two_over_G = double(d.P.two_over_G);
  chk.status = b->d_status + i;
  double *ux = nullptr, *uy = nullptr;
  if (at_rest) {
    ux = b->d_tmp + cells;
    uy = b->d_tmp + 2 * cells;
    LBM_BCUDA(b, rest_velocity_launch(b->d_tmp, d.nx, d.ny, b->p.R * b->T[i], b->p.a, b->p.b,
                                      b->p.G, ux, uy, b->d_status + i, b->stream));
    count_launches(1);
    b->stats.launches += 1;
  }
  LBM_BCUDA(b, set_state_launch(kFP32, b->buf[0] + d.off, nullptr, d.nx, d.ny, d.pitch,
                                size_t(d.pitch) * d.ny, b->d_tmp, ux, uy, nullptr, chk,
                                b->stream));
  to_float_kernel<<<256, 256, 0, b->stream>>>(b->d_tmp, b->snap + d.coff, cells);
  LBM_BCUDA(b, cudaGetLastError());
  count_launches(2);
  b->stats.launches += 2;
  LBM_BCUDA(b, cudaMemcpyAsync(b->h_status + i, b->d_status + i, sizeof(unsigned),
                               cudaMemcpyDeviceToHost, b->stream));
  LBM_BCUDA(b, cudaStreamSynchronize(b->stream));
  if (b->h_status[i] & kStatusInvalidInitFlag) {
    cudaMemsetAsync(b->d_status + i, 0, sizeof(unsigned), b->stream);
    cudaStreamSynchronize(b->stream);
    return bfail(b, LBM_E_INVAL, "rho of instance " + std::to_string(i) +
                                     " outside the domain of psi");
  }
  // a restart: the instance runs again from this state; its step count keeps
  // the steps already spent
  b->fresh[i] = 1;
  b->conv[i] = ConvState{};
  b->res[i].status = LBM_RUN_ACTIVE;
  if (std::find(b->active.begin(), b->active.end(), i) == b->active.end()) {
    b->active.push_back(i);
    std::sort(b->active.begin(), b->active.end());
    b->stats.n_active = int(b->active.size());
  }
  b->initialized = true;
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_init_density(lbm_batch* b, int i, const double* rho) {
  return batch_init_state(b, i, rho, false);
}

lbm_status lbm_batch_init_density_at_rest(lbm_batch* b, int i, const double* rho) {
  return batch_init_state(b, i, rho, true);
}

lbm_status lbm_batch_init_slabs(lbm_batch* b, const double* rho_g, const double* rho_l,
                                const double* width) {
  if (!b || !rho_g || !rho_l || !width) return bfail(b, LBM_E_INVAL, "null argument");
  BDeviceGuard guard(b->p.device);
  std::vector<double> prof(3 * b->count);
  for (int i = 0; i < b->count; ++i) {
    prof[3 * i] = rho_g[i];
    prof[3 * i + 1] = rho_l[i];
    prof[3 * i + 2] = width[i];
  }
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_prof, prof.data(), prof.size() * sizeof(double),
                               cudaMemcpyHostToDevice, b->stream));
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_inst, b->desc.data(), b->count * sizeof(BatchInst),
                               cudaMemcpyHostToDevice, b->stream));
  LBM_BCUDA(b, cudaMemsetAsync(b->d_status, 0, b->count * sizeof(unsigned), b->stream));
  dim3 grid(64, b->count);
  batch_init_slab_kernel<<<grid, 256, 0, b->stream>>>(b->d_inst, b->d_prof, b->buf[0], b->snap,
                                                       b->d_status);
  LBM_BCUDA(b, cudaGetLastError());
  count_launches(1);
  b->stats.launches += 1;
  LBM_BCUDA(b, cudaMemcpyAsync(b->h_status, b->d_status, b->count * sizeof(unsigned),
                               cudaMemcpyDeviceToHost, b->stream));
  LBM_BCUDA(b, cudaStreamSynchronize(b->stream));  // prof is a local vector
  for (int i = 0; i < b->count; ++i)
    if (b->h_status[i] & kStatusInvalidInitFlag) {
      cudaMemsetAsync(b->d_status, 0, b->count * sizeof(unsigned), b->stream);
      cudaStreamSynchronize(b->stream);
      return bfail(b, LBM_E_INVAL, "slab of instance " + std::to_string(i) +
                                       " outside the domain of psi");
    }
  for (int i = 0; i < b->count; ++i) {
    b->fresh[i] = 1;
    b->conv[i] = ConvState{};
    b->res[i] = lbm_result{};
  }
  b->active.resize(b->count);
  std::iota(b->active.begin(), b->active.end(), 0);
  b->stats.n_active = b->count;
  b->initialized = true;
  return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch* b, int max_windows, int* n_active) {
  if (!b || max_windows < 0) return bfail(b, LBM_E_INVAL, "bad argument");
  if (!b->initialized) return bfail(b, LBM_E_STATE, "batch not initialised");
  BDeviceGuard guard(b->p.device);
  for (int w = 0; w < max_windows && !b->active.empty(); ++w) {
    int mode = LBM_BATCH_WORKLIST, rows = 32;
    choose_config(b, mode, rows);
    for (auto& d : b->desc) set_geometry(d, rows > 0 ? rows : 32);
    lbm_status st = upload_tables(b, mode);
    if (st != LBM_OK) return st;
    cudaGraphExec_t g = nullptr;
    st = window_graph(b, mode, &g);
    if (st != LBM_OK && mode == LBM_BATCH_COOPERATIVE && b->p.mode == LBM_BATCH_AUTO) {
      // cooperative windows unavailable here: drop them and use the work list
      b->coop_grid = 0;
      b->tuner.disable(LBM_BATCH_COOPERATIVE);
      mode = LBM_BATCH_WORKLIST;
      st = window_graph(b, mode, &g);
    }
    if (st != LBM_OK) return st;
    const size_t cells = active_cells(b);
    LBM_BCUDA(b, cudaEventRecord(b->ev0, b->stream));
    LBM_BCUDA(b, cudaGraphLaunch(g, b->stream));
    LBM_BCUDA(b, cudaEventRecord(b->ev1, b->stream));
    // two class kernels per step (work list) or per window (persistent), and
    // the reduction
    // (one cooperative kernel per window)
    const unsigned long long kernels =
        mode == LBM_BATCH_COOPERATIVE
            ? 1
            : (class_grid(b, mode, 0) > 0 ? 1 : 0) + (class_grid(b, mode, 1) > 0 ? 1 : 0);
    const bool per_step = mode == LBM_BATCH_WORKLIST || mode == LBM_BATCH_WORKLIST_DYNAMIC ||
                          mode == LBM_BATCH_BALANCED;
    const unsigned long long nl = (per_step ? kernels * b->p.window : kernels) + 1;
    count_launches(nl);
    b->stats.launches += nl;
    LBM_BCUDA(b, cudaMemcpyAsync(b->h_out, b->d_out, b->count * sizeof(BatchOut),
                                 cudaMemcpyDeviceToHost, b->stream));
    LBM_BCUDA(b, cudaMemcpyAsync(b->h_status, b->d_status, b->count * sizeof(unsigned),
                                 cudaMemcpyDeviceToHost, b->stream));
    LBM_BCUDA(b, cudaStreamSynchronize(b->stream));
    if (mode == LBM_BATCH_COOPERATIVE) {
      unsigned sync_err = 0;
      LBM_BCUDA(b, cudaMemcpy(&sync_err, b->d_sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
      if (sync_err) return bfail(b, LBM_E_TIMEOUT, "grid barrier of a cooperative window gave up");
    }
    float ms = 0.f;
    LBM_BCUDA(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    b->stats.gpu_ms += ms;
    b->stats.windows += 1;
    b->stats.mode = mode;
    b->stats.rows_per_item = rows;
    if (b->p.mode == LBM_BATCH_AUTO)
      b->tuner.record(mode, rows, ms * 1e6 / (double(cells) * b->p.window));
    std::vector<int> still;
    const ConvRule rule{b->p.conv,   b->p.tol,       b->p.conv_rel,
                        b->p.window, b->p.max_steps, b->p.trend_tol};
    for (int i : b->active) {
      const BatchOut& o = b->h_out[i];
      WindowObs obs;
      obs.rho_g = o.rho_g;
      obs.rho_l = o.rho_l;
      obs.width = o.width;
      obs.mass = o.mass;
      obs.max_abs = o.max_abs;
      obs.max_dev = o.max_dev;
      obs.finite = o.finite != 0;
      obs.diverged = (b->h_status[i] & kStatusDivergedFlag) != 0;
      const bool first = b->fresh[i] != 0;
      b->fresh[i] = 0;
      lbm_result& r = b->res[i];
      r.status = window_verdict(rule, obs, first, b->conv[i], r);
      if (r.status == LBM_RUN_ACTIVE) still.push_back(i);
    }
    b->active.swap(still);
    b->stats.n_active = int(b->active.size());
  }
  if (n_active) *n_active = int(b->active.size());
  return LBM_OK;
}

lbm_status lbm_batch_get_result(const lbm_batch* b, int i, lbm_result* r) {
  if (!b || !r || i < 0 || i >= b->count) return LBM_E_INVAL;
  *r = b->res[i];
  return LBM_OK;
}

lbm_status lbm_batch_get_density(lbm_batch* b, int i, double* rho) {
  if (!b || !rho || i < 0 || i >= b->count) return bfail(b, LBM_E_INVAL, "bad argument");
  if (!b->initialized) return bfail(b, LBM_E_STATE, "batch not initialised");
  BDeviceGuard guard(b->p.device);
  const size_t cells = size_t(b->desc[i].nx) * b->desc[i].ny;
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_inst, b->desc.data(), b->count * sizeof(BatchInst),
                               cudaMemcpyHostToDevice, b->stream));
  batch_density_kernel<<<128, 256, 0, b->stream>>>(b->d_inst, i, b->buf[0], b->d_tmp);
  LBM_BCUDA(b, cudaGetLastError());
  count_launches(1);
  LBM_BCUDA(b, cudaMemcpyAsync(rho, b->d_tmp, cells * sizeof(double), cudaMemcpyDeviceToHost,
                               b->stream));
  LBM_BCUDA(b, cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

lbm_status lbm_batch_get_moments(lbm_batch* b, int i, double* rho, double* vx, double* vy) {
  if (!b || i < 0 || i >= b->count) return bfail(b, LBM_E_INVAL, "bad argument");
  if (!b->initialized) return bfail(b, LBM_E_STATE, "batch not initialised");
  BDeviceGuard guard(b->p.device);
  const BatchInst& d = b->desc[i];
  const size_t cells = size_t(d.nx) * d.ny;
  LBM_BCUDA(b, cudaMemcpyAsync(b->d_inst, b->desc.data(), b->count * sizeof(BatchInst),
                               cudaMemcpyHostToDevice, b->stream));
  const int items = ((d.nx + 31) / 32) * ((d.ny + 7) / 8);
  const int grid = (items + kWorklistThreads / 32 - 1) / (kWorklistThreads / 32);
  double* o = b->d_tmp;
  if (d.scheme == LBM_SCHEME_NOFORCE)
    batch_observe_kernel<kModeObserveNoForce><<<grid, kWorklistThreads, 0, b->stream>>>(
        b->d_inst, i, b->buf[0], o, o + cells, o + 2 * cells, b->d_status);
  else
    batch_observe_kernel<kModeObserve><<<grid, kWorklistThreads, 0, b->stream>>>(
        b->d_inst, i, b->buf[0], o, o + cells, o + 2 * cells, b->d_status);
  LBM_BCUDA(b, cudaGetLastError());
  count_launches(1);
  double* host[3] = {rho, vx, vy};
  for (int k = 0; k < 3; ++k)
    if (host[k])
      LBM_BCUDA(b, cudaMemcpyAsync(host[k], o + k * cells, cells * sizeof(double),
                                   cudaMemcpyDeviceToHost, b->stream));
  LBM_BCUDA(b, cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

lbm_status lbm_selftest_grid_barrier_timeout(int device, int* result) {
  if (!result) return LBM_E_INVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return LBM_E_CUDA;
  }
  BDeviceGuard guard(device);
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop)
    return LBM_E_CUDA;
  unsigned* d_sync = nullptr;
  if (cudaMalloc(&d_sync, 3 * sizeof(unsigned)) != cudaSuccess) return LBM_E_NOMEM;
  lbm_status st = LBM_OK;
  unsigned h[3] = {0, 0, 0};
  void* args[] = {&d_sync};
  if (cudaMemset(d_sync, 0, 3 * sizeof(unsigned)) != cudaSuccess ||
      cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(barrier_selftest_kernel),
                                  dim3(4), dim3(32), args, 0, nullptr) != cudaSuccess ||
      cudaMemcpy(h, d_sync, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    st = LBM_E_CUDA;
  }
  count_launches(1);
  cudaFree(d_sync);
  if (st == LBM_OK) *result = (h[2] & kStatusTimeout) ? LBM_E_TIMEOUT : LBM_OK;
  return st;
}

lbm_status lbm_batch_get_stats(const lbm_batch* b, lbm_batch_stats* s) {
  if (!b || !s) return LBM_E_INVAL;
  *s = b->stats;
  return LBM_OK;
}

}  // extern "C"
