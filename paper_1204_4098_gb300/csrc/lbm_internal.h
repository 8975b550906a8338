// Internal interface between the C-ABI layer (lbm_capi.cu) and the kernel
// translation units (one per storage precision, compiled in parallel).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace lbm {

// Type-erased arguments of the warp-strip step / observe kernel.
struct StripLaunch {
  const void* src;
  void* dst;
  const float* rho_src;
  float* rho_dst;
  double* out_rho;
  double* out_vx;
  double* out_vy;
  unsigned* status;
  int nx, ny;                  // ny: rows of the buffers
  int y_begin, y_end;          // rows computed
  int out_row0;                // observe mode: buffer row of output row 0
  int n_strips, band_rows, n_bands;
  size_t plane;
  // physics (converted to the compute type by each translation unit)
  double RT, a, b4, two_over_G, minus_G, tau, omega, sigma_ups, guo;
  double s_e, s_eps, s_q;  // MRT rates (scheme 6)
};

enum Precision { kFP32 = 0, kFP64 = 1, kBF16Dev = 2, kFP16Dev = 3 };
enum Mode { kStepMode = 0, kObserveMode = 1, kObserveNoForceMode = 2 };

constexpr int kStripCtaThreads = 128;

// device status word bits
constexpr unsigned kStatusDivergedFlag = 1u;
constexpr unsigned kStatusTimeoutFlag = 2u;
constexpr unsigned kStatusInvalidInitFlag = 4u;

// Equation-of-state constants for the initial-density domain check.
struct EosCheck {
  double RT, a, b4, two_over_G;
  unsigned* status;  // NULL: no check
};

// Warp-strip kernel of the given precision / scheme / mode on `grid` CTAs.
cudaError_t strip_launch(int precision, int scheme, int mode, const StripLaunch& L,
                         int grid, cudaStream_t s);
// Resident CTAs per SM of that kernel.
cudaError_t strip_occupancy(int precision, int scheme, int mode, int* blocks_per_sm);
// Two-columns-per-lane kernel (direct storage FP32 / FP64; needs even nx;
// L.n_strips counts 64-column strips).
cudaError_t strip2_launch(int precision, int scheme, int mode, const StripLaunch& L, int grid,
                          cudaStream_t s);
cudaError_t strip2_occupancy(int precision, int scheme, int mode, int* blocks_per_sm);
// Bulk-copy staged step kernel (FP32 only; needs nx % 4 == 0 and nx >= 64).
cudaError_t strip_tma_launch(int precision, int scheme, const StripLaunch& L, int grid,
                             cudaStream_t s);
cudaError_t strip_tma_occupancy(int precision, int scheme, int* blocks_per_sm);

// f*_a(x') = f_a(x' + e_a) from f_eq(rho, u) (f_in == NULL) or from f_in;
// with f_in == NULL and chk.status set, flags rho outside the domain of psi.
// dst rows have `pitch` >= nx elements (columns past nx: copies of columns
// (x - nx) mod nx); plane = pitch * ny; rho, ux, uy, f_in are unpadded.
cudaError_t set_state_launch(int precision, void* dst, float* rho_dst, int nx, int ny,
                             int pitch, size_t plane, const double* rho, const double* ux,
                             const double* uy, const double* f_in, const EosCheck& chk,
                             cudaStream_t s);
// u = -F / (2 rho) at every cell, F the force of Eq. 3 on the device density
// field rho (FP64): the velocity whose equilibrium is at rest, i.e. has zero
// actual velocity v = u + F / (2 rho) (Table I).  Cells outside the domain of
// psi get u = 0 and set kStatusInvalidInitFlag in *status (if non-NULL).
cudaError_t rest_velocity_launch(const double* rho, int nx, int ny, double RT, double a,
                                 double b, double G, double* ux, double* uy, unsigned* status,
                                 cudaStream_t s);
// f_a(x, t) = f*_a(x - e_a) into f_out (FP64).
cudaError_t get_state_launch(int precision, const void* src, const float* rho_src, int nx,
                             int ny, size_t plane, double* f_out, cudaStream_t s);
// Sum of the populations of cells [first, first + count) of every plane in
// FP64: partial sums into `partial` (n_partial doubles of scratch), then the
// total into *out (device pointer).
cudaError_t mass_launch(int precision, const void* src, const float* rho_src, size_t plane,
                        size_t first, size_t count, double* partial, int n_partial,
                        double* out, cudaStream_t s);

size_t storage_bytes(int precision);  // bytes per population

// Counts kernel launches queued by the library (for benchmark accounting).
void count_launches(unsigned long long n);

}  // namespace lbm
