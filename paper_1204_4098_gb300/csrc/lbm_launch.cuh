// Launch helpers shared by the per-precision kernel translation units.
#pragma once

#include <type_traits>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

template <class S>
StripArgs<S> make_args(const StripLaunch& L) {
  using C = typename S::C;
  StripArgs<S> A;
  A.src = static_cast<const typename S::T*>(L.src);
  A.dst = static_cast<typename S::T*>(L.dst);
  A.rho_src = L.rho_src;
  A.rho_dst = L.rho_dst;
  A.out_rho = L.out_rho;
  A.out_vx = L.out_vx;
  A.out_vy = L.out_vy;
  A.status = L.status;
  A.nx = L.nx;
  A.ny = L.ny;
  A.pitch = L.nx;  // the single-lattice buffers are unpadded
  A.y_begin = L.y_begin;
  A.y_end = L.y_end;
  A.out_row0 = L.out_row0;
  A.n_strips = L.n_strips;
  A.band_rows = L.band_rows;
  A.n_bands = L.n_bands;
  A.plane = L.plane;
  A.P.RT = C(L.RT);
  A.P.a = C(L.a);
  A.P.b4 = C(L.b4);
  A.P.two_over_G = C(L.two_over_G);
  A.P.minus_G = C(L.minus_G);
  A.P.tau = C(L.tau);
  A.P.omega = C(L.omega);
  A.P.sigma_ups = C(L.sigma_ups);
  A.P.guo = C(L.guo);
  A.P.scheme = 0;  // the single-domain kernels fix the scheme at compile time
  A.P.s_e = C(L.s_e);
  A.P.s_eps = C(L.s_eps);
  A.P.s_q = C(L.s_q);
  return A;
}

template <class S, int SCHEME, int MODE>
cudaError_t launch_one(const StripLaunch& L, int grid, cudaStream_t s) {
  strip_kernel<S, SCHEME, MODE><<<grid, kStripThreads, 0, s>>>(make_args<S>(L));
  return cudaGetLastError();
}

template <class S, int SCHEME, int MODE>
cudaError_t occ_one(int* b) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, strip_kernel<S, SCHEME, MODE>,
                                                       kStripThreads, 0);
}

// scheme x mode dispatch for one storage type
template <class S>
cudaError_t strip_launch_t(int scheme, int mode, const StripLaunch& L, int grid,
                           cudaStream_t s) {
  if (mode == kObserveMode) return launch_one<S, kSC, kModeObserve>(L, grid, s);
  if (mode == kObserveNoForceMode) return launch_one<S, kSC, kModeObserveNoForce>(L, grid, s);
  switch (scheme) {
    case kSC: return launch_one<S, kSC, kModeStep>(L, grid, s);
    case kEDM: return launch_one<S, kEDM, kModeStep>(L, grid, s);
    case kImproved: return launch_one<S, kImproved, kModeStep>(L, grid, s);
    case kNoForce: return launch_one<S, kNoForce, kModeStep>(L, grid, s);
    case kEDMMod: return launch_one<S, kEDMMod, kModeStep>(L, grid, s);
    case kLadd: return launch_one<S, kLadd, kModeStep>(L, grid, s);
    case kMRT: return launch_one<S, kMRT, kModeStep>(L, grid, s);
  }
  return cudaErrorInvalidValue;
}

template <class S>
cudaError_t strip_occupancy_t(int scheme, int mode, int* b) {
  if (mode == kObserveMode) return occ_one<S, kSC, kModeObserve>(b);
  if (mode == kObserveNoForceMode) return occ_one<S, kSC, kModeObserveNoForce>(b);
  switch (scheme) {
    case kSC: return occ_one<S, kSC, kModeStep>(b);
    case kEDM: return occ_one<S, kEDM, kModeStep>(b);
    case kImproved: return occ_one<S, kImproved, kModeStep>(b);
    case kNoForce: return occ_one<S, kNoForce, kModeStep>(b);
    case kEDMMod: return occ_one<S, kEDMMod, kModeStep>(b);
    case kLadd: return occ_one<S, kLadd, kModeStep>(b);
    case kMRT: return occ_one<S, kMRT, kModeStep>(b);
  }
  return cudaErrorInvalidValue;
}

// Bulk-copy staged step kernel: FP32 direct storage only.
template <class S>
cudaError_t strip_tma_launch_t(int scheme, const StripLaunch& L, int grid, cudaStream_t s) {
  if constexpr (!std::is_same<S, StoreF32>::value) {
    return cudaErrorNotSupported;
  } else {
    const StripArgs<S> A = make_args<S>(L);
    switch (scheme) {
      case kSC: strip_tma_kernel<kSC><<<grid, kStripThreads, 0, s>>>(A); break;
      case kEDM: strip_tma_kernel<kEDM><<<grid, kStripThreads, 0, s>>>(A); break;
      case kImproved: strip_tma_kernel<kImproved><<<grid, kStripThreads, 0, s>>>(A); break;
      case kNoForce: strip_tma_kernel<kNoForce><<<grid, kStripThreads, 0, s>>>(A); break;
      case kEDMMod: strip_tma_kernel<kEDMMod><<<grid, kStripThreads, 0, s>>>(A); break;
      case kLadd: strip_tma_kernel<kLadd><<<grid, kStripThreads, 0, s>>>(A); break;
      case kMRT: strip_tma_kernel<kMRT><<<grid, kStripThreads, 0, s>>>(A); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
}

template <class S>
cudaError_t strip_tma_occupancy_t(int scheme, int* b) {
  if constexpr (!std::is_same<S, StoreF32>::value) {
    return cudaErrorNotSupported;
  } else {
    switch (scheme) {
      case kSC: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, strip_tma_kernel<kSC>, kStripThreads, 0);
      case kEDM: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, strip_tma_kernel<kEDM>, kStripThreads, 0);
      case kImproved: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, strip_tma_kernel<kImproved>, kStripThreads, 0);
      case kNoForce: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, strip_tma_kernel<kNoForce>, kStripThreads, 0);
      case kEDMMod: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, strip_tma_kernel<kEDMMod>, kStripThreads, 0);
      case kLadd: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, strip_tma_kernel<kLadd>, kStripThreads, 0);
      case kMRT: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, strip_tma_kernel<kMRT>, kStripThreads, 0);
    }
    return cudaErrorInvalidValue;
  }
}

// Two-columns-per-lane kernel (every storage type; needs even nx).
template <class S, int SCHEME, int MODE>
cudaError_t launch2_one(const StripLaunch& L, int grid, cudaStream_t s) {
  strip2_kernel<S, SCHEME, MODE><<<grid, kStripThreads, 0, s>>>(make_args<S>(L));
  return cudaGetLastError();
}
template <class S, int SCHEME, int MODE>
cudaError_t occ2_one(int* b) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, strip2_kernel<S, SCHEME, MODE>,
                                                       kStripThreads, 0);
}
template <class S>
cudaError_t strip2_launch_t(int scheme, int mode, const StripLaunch& L, int grid,
                            cudaStream_t s) {
  {
    if (mode == kObserveMode) return launch2_one<S, kSC, kModeObserve>(L, grid, s);
    if (mode == kObserveNoForceMode) return launch2_one<S, kSC, kModeObserveNoForce>(L, grid, s);
    switch (scheme) {
      case kSC: return launch2_one<S, kSC, kModeStep>(L, grid, s);
      case kEDM: return launch2_one<S, kEDM, kModeStep>(L, grid, s);
      case kImproved: return launch2_one<S, kImproved, kModeStep>(L, grid, s);
      case kNoForce: return launch2_one<S, kNoForce, kModeStep>(L, grid, s);
      case kEDMMod: return launch2_one<S, kEDMMod, kModeStep>(L, grid, s);
      case kLadd: return launch2_one<S, kLadd, kModeStep>(L, grid, s);
      case kMRT: return launch2_one<S, kMRT, kModeStep>(L, grid, s);
    }
    return cudaErrorInvalidValue;
  }
}
template <class S>
cudaError_t strip2_occupancy_t(int scheme, int mode, int* b) {
  {
    if (mode == kObserveMode) return occ2_one<S, kSC, kModeObserve>(b);
    if (mode == kObserveNoForceMode) return occ2_one<S, kSC, kModeObserveNoForce>(b);
    switch (scheme) {
      case kSC: return occ2_one<S, kSC, kModeStep>(b);
      case kEDM: return occ2_one<S, kEDM, kModeStep>(b);
      case kImproved: return occ2_one<S, kImproved, kModeStep>(b);
      case kNoForce: return occ2_one<S, kNoForce, kModeStep>(b);
      case kEDMMod: return occ2_one<S, kEDMMod, kModeStep>(b);
      case kLadd: return occ2_one<S, kLadd, kModeStep>(b);
      case kMRT: return occ2_one<S, kMRT, kModeStep>(b);
    }
    return cudaErrorInvalidValue;
  }
}

inline int grid_for(size_t n, int threads) {
  size_t g = (n + threads - 1) / threads;
  if (g > 65535u * 8u) g = 65535u * 8u;
  return int(g < 1 ? 1 : g);
}

template <class S>
cudaError_t set_state_t(void* dst, float* rho_dst, int nx, int ny, int pitch, size_t plane,
                        const double* rho, const double* ux, const double* uy,
                        const double* f_in, const EosCheck& chk, cudaStream_t s) {
  Phys<double> P{};
  P.RT = chk.RT;
  P.a = chk.a;
  P.b4 = chk.b4;
  P.two_over_G = chk.two_over_G;
  set_state_kernel<S><<<grid_for(plane, 256), 256, 0, s>>>(
      static_cast<typename S::T*>(dst), rho_dst, nx, ny, pitch, plane, rho, ux, uy, f_in, P,
      chk.status);
  return cudaGetLastError();
}

template <class S>
cudaError_t get_state_t(const void* src, const float* rho_src, int nx, int ny, size_t plane,
                        double* f_out, cudaStream_t s) {
  get_state_kernel<S><<<grid_for(plane, 256), 256, 0, s>>>(
      static_cast<const typename S::T*>(src), rho_src, nx, ny, plane, f_out);
  return cudaGetLastError();
}

template <class S>
cudaError_t mass_t(const void* src, const float* rho_src, size_t plane, size_t first,
                   size_t count, double* partial, int n_partial, double* out, cudaStream_t s) {
  mass_partial_kernel<S><<<n_partial, kReduceThreads, 0, s>>>(
      static_cast<const typename S::T*>(src), rho_src, plane, first, count, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_partials_kernel<<<1, kReduceThreads, 0, s>>>(partial, n_partial, out);
  return cudaGetLastError();
}

}  // namespace lbm

// Defines the per-precision entry points of one translation unit.
#define LBM_DEFINE_PRECISION(SUFFIX, STORE)                                              \
  namespace lbm {                                                                       \
  cudaError_t strip_launch_##SUFFIX(int scheme, int mode, const StripLaunch& L, int grid, \
                                    cudaStream_t s) {                                   \
    return strip_launch_t<STORE>(scheme, mode, L, grid, s);                             \
  }                                                                                     \
  cudaError_t strip_occupancy_##SUFFIX(int scheme, int mode, int* b) {                  \
    return strip_occupancy_t<STORE>(scheme, mode, b);                                   \
  }                                                                                     \
  cudaError_t strip2_launch_##SUFFIX(int scheme, int mode, const StripLaunch& L, int grid, \
                                     cudaStream_t s) {                                  \
    return strip2_launch_t<STORE>(scheme, mode, L, grid, s);                            \
  }                                                                                     \
  cudaError_t strip2_occupancy_##SUFFIX(int scheme, int mode, int* b) {                 \
    return strip2_occupancy_t<STORE>(scheme, mode, b);                                  \
  }                                                                                     \
  cudaError_t strip_tma_launch_##SUFFIX(int scheme, const StripLaunch& L, int grid,      \
                                        cudaStream_t s) {                               \
    return strip_tma_launch_t<STORE>(scheme, L, grid, s);                               \
  }                                                                                     \
  cudaError_t strip_tma_occupancy_##SUFFIX(int scheme, int* b) {                        \
    return strip_tma_occupancy_t<STORE>(scheme, b);                                     \
  }                                                                                     \
  cudaError_t set_state_##SUFFIX(void* dst, float* rd, int nx, int ny, int pitch,       \
                                 size_t plane, const double* rho, const double* ux,     \
                                 const double* uy, const double* f_in,                 \
                                 const EosCheck& chk, cudaStream_t s) {                 \
    return set_state_t<STORE>(dst, rd, nx, ny, pitch, plane, rho, ux, uy, f_in, chk, s); \
  }                                                                                     \
  cudaError_t get_state_##SUFFIX(const void* src, const float* rs, int nx, int ny,       \
                                 size_t plane, double* f_out, cudaStream_t s) {         \
    return get_state_t<STORE>(src, rs, nx, ny, plane, f_out, s);                        \
  }                                                                                     \
  cudaError_t mass_##SUFFIX(const void* src, const float* rs, size_t plane, size_t first, \
                            size_t count, double* partial, int n_partial, double* out,  \
                            cudaStream_t s) {                                           \
    return mass_t<STORE>(src, rs, plane, first, count, partial, n_partial, out, s);      \
  }                                                                                     \
  }
