// Fused pseudopotential D2Q9 step kernels (templated on storage and scheme).
//
// One time step (Li, Luo & Li, Eq. 1) in pull form: the buffer src holds the
// post-collision populations f*_a(x', t-1) at the cells they were collided
// on; the state at time t is f_a(x, t) = f*_a(x - e_a, t - 1).  The kernel
// reads src, computes rho, u (Sec. III A), psi (Eqs. 8, 23), the force of
// Eq. 3 and the collision, and writes f*_a(x, t) to dst -- one read and one
// write of every population per step, nothing else through HBM.
//
// Work decomposition ("warp strips"): a warp owns 32 consecutive columns
// (one per lane) and a band of rows, which it marches down.  For each row it
// needs psi on the row above and below and on the two columns beside the
// strip; psi of a row is computed once, when the row is first loaded, and
// kept in registers for the three output rows that use it.  The x neighbours
// come from the adjacent lanes by shuffle, the two halo columns from one
// extra load per direction spread over lanes 0..8 and 16..24.  The next row
// is loaded while the current one is computed.  Warps of a band run side by
// side, so the halo reads of one strip hit the lines its neighbours just
// brought into L2.  Periodic wrap is applied to the indices, so any nx, ny
// >= 1 works; lanes past the right edge of a ragged strip evaluate the
// wrapped columns (serving as the right neighbour) and store nothing.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kStripWarpsPerCta = 4;
constexpr int kStripThreads = kStripWarpsPerCta * 32;
// Resident CTAs per SM the register allocation must allow (occupancy target).
#ifndef LBM_STRIP_MIN_BLOCKS
#define LBM_STRIP_MIN_BLOCKS 6
#endif
// 1: unroll the row loop by three (no register moves, more registers).
#ifndef LBM_STRIP_UNROLL3
#define LBM_STRIP_UNROLL3 0
#endif

template <class S>
struct StripArgs {
  const typename S::T* src;   // [9][ny][nx] post-collision populations (t-1)
  typename S::T* dst;         // [9][ny][nx] post-collision populations (t)
  const float* rho_src;       // deviation storage: density plane of src
  float* rho_dst;             // deviation storage: density plane of dst
  double* out_rho;            // observe mode: rho, v (FP64, [ny][nx])
  double* out_vx;
  double* out_vy;
  unsigned* status;           // device status word
  int nx, ny;
  int n_strips;               // ceil(nx / 32)
  int band_rows;              // rows per warp
  int n_bands;                // ceil(ny / band_rows)
  size_t plane;               // nx * ny
  Phys<typename S::C> P;
};

enum { kModeStep = 0, kModeObserve = 1, kModeObserveNoForce = 2 };

// Value of population a pulled from source cell index idx.  kCoherent loads
// bypass L1 (ld.global.cg): needed when the same kernel wrote the source
// buffer in an earlier step (persistent batch kernel); otherwise the
// read-only path is used.
template <class S, bool kCoherent>
__device__ __forceinline__ typename S::C pull_one(const StripArgs<S>& A, int a, int idx) {
  using C = typename S::C;
  C v;
  if constexpr (kCoherent) {
    v = S::to_c(__ldcg(A.src + a * A.plane + idx));
    if constexpr (S::kDev) v = fma_rn(w_of<C>(a), C(__ldcg(A.rho_src + idx)), v);
  } else {
    v = S::to_c(__ldg(A.src + a * A.plane + idx));
    if constexpr (S::kDev) v = fma_rn(w_of<C>(a), C(__ldg(A.rho_src + idx)), v);
  }
  return v;
}

static __constant__ int c_ex[16] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0};
static __constant__ int c_ey[16] = {0, 0, 1, 0, -1, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0};

// One warp advances (or observes) the cells of one strip x band item.
template <class S, int SCHEME, int MODE, bool kCoherent>
__device__ __forceinline__ void strip_run(const StripArgs<S>& A, int strip, int band,
                                          int lane) {
  using C = typename S::C;
  constexpr bool kNeedPsi = !(MODE == kModeObserveNoForce ||
                              (MODE == kModeStep && SCHEME == kNoForce));
  const unsigned FULL = 0xffffffffu;
  const int nx = A.nx, ny = A.ny;
  const int y0 = band * A.band_rows;
  const int y1 = min(y0 + A.band_rows, ny);

  const int x = strip * 32 + lane;
  const bool active = x < nx;
  const int c = x % nx;
  const int cm = c == 0 ? nx - 1 : c - 1;
  const int cp = c == nx - 1 ? 0 : c + 1;
  // halo lanes: 0..8 pull direction `lane` at the column left of the strip,
  // 16..24 direction `lane - 16` at the column right of it
  const int ha = lane & 15;
  const int hcol = lane < 16 ? (strip * 32 - 1 + nx) % nx : (strip * 32 + 32) % nx;
  const int hex = c_ex[ha], hey = c_ey[ha];
  const int hsx = ((hcol - hex) % nx + nx) % nx;
  const bool hlane = ha < kQ;
  const int hbase = lane & 16;

  bool bad = false;

  // pulled populations of row y at this lane's column, plus this lane's halo value
  auto load_row = [&](int y, C (&P)[kQ], C& h) {
    const int ym = y == 0 ? ny - 1 : y - 1;
    const int yp = y == ny - 1 ? 0 : y + 1;
    const int r0 = y * nx, rm = ym * nx, rp = yp * nx;
    P[0] = pull_one<S, kCoherent>(A, 0, r0 + c);
    P[1] = pull_one<S, kCoherent>(A, 1, r0 + cm);
    P[2] = pull_one<S, kCoherent>(A, 2, rm + c);
    P[3] = pull_one<S, kCoherent>(A, 3, r0 + cp);
    P[4] = pull_one<S, kCoherent>(A, 4, rp + c);
    P[5] = pull_one<S, kCoherent>(A, 5, rm + cm);
    P[6] = pull_one<S, kCoherent>(A, 6, rm + cp);
    P[7] = pull_one<S, kCoherent>(A, 7, rp + cp);
    P[8] = pull_one<S, kCoherent>(A, 8, rp + cm);
    if constexpr (kNeedPsi) {
      int hy = y - hey;  // |hey| <= 1 and 0 <= y < ny: one conditional wrap
      hy = hy < 0 ? hy + ny : (hy >= ny ? hy - ny : hy);
      h = hlane ? pull_one<S, kCoherent>(A, ha, hy * nx + hsx) : C(0);
    }
  };
  // density with a fixed summation order (the halo path below repeats it)
  auto rho_of = [](const C (&P)[kQ]) {
    C r = P[0];
#pragma unroll
    for (int a = 1; a < kQ; ++a) r = add_rn(r, P[a]);
    return r;
  };
  // psi of the halo column of this lane's half-warp
  auto halo_psi = [&](C h) {
    C r = __shfl_sync(FULL, h, hbase);
#pragma unroll
    for (int a = 1; a < kQ; ++a) r = add_rn(r, __shfl_sync(FULL, h, hbase + a));
    return psi_of_rho(r, A.P, bad);
  };

  // psi ring: rows y-1 (m), y (z), y+1 (p); W / C / E = columns x-1, x, x+1
  C Wm = 0, Cm = 0, Em = 0, Wz = 0, Cz = 0, Ez = 0;
  C rho0;

  auto psi_row = [&](const C (&P)[kQ], C h, C& Wv, C& Cv, C& Ev, C& rho_out) {
    rho_out = rho_of(P);
    if constexpr (kNeedPsi) {
      Cv = psi_of_rho(rho_out, A.P, bad);
      const C hp = halo_psi(h);
      Wv = __shfl_up_sync(FULL, Cv, 1);
      Ev = __shfl_down_sync(FULL, Cv, 1);
      if (lane == 0) Wv = hp;
      if (lane == 31) Ev = hp;
    }
  };

  // Output row y: Pcur holds its pulled populations, Pnext (with halo hnext)
  // those of row y + 1, and row y + 2 is loaded into Pload while this row is
  // computed.  The three buffers rotate through the unrolled loop below, so
  // no populations are copied between registers.
  auto row = [&](int y, C (&Pcur)[kQ], const C (&Pnext)[kQ], C hnext, C (&Pload)[kQ],
                 C& hload) {
    if (y + 2 <= y1) load_row(y + 2 >= ny ? y + 2 - ny : y + 2, Pload, hload);
    C Wp = 0, Cp = 0, Ep = 0, rho1;
    psi_row(Pnext, hnext, Wp, Cp, Ep, rho1);

    C Fx = C(0), Fy = C(0);
    if constexpr (kNeedPsi) {
      // Eq. 3: F = -G psi(x) sum_a w(|e_a|^2) psi(x + e_a) e_a
      const C third = C(1) / C(3), twelfth = C(1) / C(12);
      const C sx = fma_rn(third, sub_rn(Ez, Wz),
                          mul_rn(twelfth, add_rn(sub_rn(Ep, Wp), sub_rn(Em, Wm))));
      const C sy = fma_rn(third, sub_rn(Cp, Cm),
                          mul_rn(twelfth, sub_rn(add_rn(Ep, Wp), add_rn(Em, Wm))));
      const C gpsi = mul_rn(A.P.minus_G, Cz);
      Fx = mul_rn(gpsi, sx);
      Fy = mul_rn(gpsi, sy);
    }

    const int idx = y * nx + c;
    if constexpr (MODE == kModeStep) {
      collide<C, SCHEME>(Pcur, rho0, Fx, Fy, Cz, A.P);
      if (active) {
        if constexpr (S::kDev) {
          // the density plane absorbs the 16-bit rounding of the deviations,
          // so w_a rho_dst + d_a still sums to rho over a (mass conserved)
          C resid = rho0;
#pragma unroll
          for (int a = 0; a < kQ; ++a) {
            const typename S::T d = S::from_c(sub_rn(Pcur[a], mul_rn(w_of<C>(a), rho0)));
            A.dst[a * A.plane + idx] = d;
            resid = sub_rn(resid, S::to_c(d));
          }
          A.rho_dst[idx] = float(resid);
        } else {
#pragma unroll
          for (int a = 0; a < kQ; ++a) A.dst[a * A.plane + idx] = S::from_c(Pcur[a]);
        }
      }
    } else {
      if (active) {
        const C jx = (Pcur[1] - Pcur[3]) + (Pcur[5] - Pcur[6]) + (Pcur[8] - Pcur[7]);
        const C jy = (Pcur[2] - Pcur[4]) + (Pcur[5] + Pcur[6]) - (Pcur[7] + Pcur[8]);
        const double r = double(rho0);
        A.out_rho[idx] = r;
        A.out_vx[idx] = (double(jx) + 0.5 * double(Fx)) / r;
        A.out_vy[idx] = (double(jy) + 0.5 * double(Fy)) / r;
      }
    }
    Wm = Wz; Cm = Cz; Em = Ez;
    Wz = Wp; Cz = Cp; Ez = Ep;
    rho0 = rho1;
  };

  C PA[kQ], PB[kQ], PC[kQ];
  C hA = C(0), hB = C(0), hC = C(0);
  // prologue: psi of rows y0 - 1 and y0, populations of y0 (PA) and y0 + 1 (PB)
  {
    C rdummy;
    load_row(y0 == 0 ? ny - 1 : y0 - 1, PA, hA);
    psi_row(PA, hA, Wm, Cm, Em, rdummy);
    load_row(y0, PA, hA);
    psi_row(PA, hA, Wz, Cz, Ez, rho0);
    load_row(y0 + 1 == ny ? 0 : y0 + 1, PB, hB);
  }
#if LBM_STRIP_UNROLL3
  int y = y0;
  for (; y + 3 <= y1; y += 3) {
    row(y, PA, PB, hB, PC, hC);
    row(y + 1, PB, PC, hC, PA, hA);
    row(y + 2, PC, PA, hA, PB, hB);
  }
  if (y < y1) {
    row(y, PA, PB, hB, PC, hC);
    if (y + 1 < y1) row(y + 1, PB, PC, hC, PA, hA);
  }
#else
  // rolled loop: the three population buffers are copied down once per row,
  // which costs moves but keeps the register count (occupancy) lower
  for (int y = y0; y < y1; ++y) {
    row(y, PA, PB, hB, PC, hC);
#pragma unroll
    for (int a = 0; a < kQ; ++a) { PA[a] = PB[a]; PB[a] = PC[a]; }
    hB = hC;
  }
#endif
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(A.status, kStatusDiverged);
}

template <class S, int SCHEME, int MODE>
__global__ void __launch_bounds__(kStripThreads, LBM_STRIP_MIN_BLOCKS)
strip_kernel(const StripArgs<S> A) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * kStripThreads + threadIdx.x) >> 5;
  const int strip = gwarp % A.n_strips;
  const int band = gwarp / A.n_strips;
  if (band >= A.n_bands) return;  // warp-uniform
  strip_run<S, SCHEME, MODE, false>(A, strip, band, lane);
}

// ---------------------------------------------------------------------------
// initialisation and checkpoint kernels (not on the per-step path)
// ---------------------------------------------------------------------------

// f*_a(x') = f_a(x' + e_a): store a physical state (time t, before the pull)
// so that the next pull reproduces it.  The physical state is either
// f_eq(rho, u) (init) or given populations (set).
template <class S>
__global__ void set_state_kernel(typename S::T* dst, float* rho_dst, int nx, int ny,
                                 size_t plane, const double* rho, const double* ux,
                                 const double* uy, const double* f_in, Phys<double> P,
                                 unsigned* status) {
  const size_t n = plane;
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = int(i % nx), y = int(i / nx);
    if (!f_in && status) (void)psi_of_rho(rho[i], P, bad);  // domain of psi at the start
    double fs[kQ];
    double rsum = 0.0;
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const int xd = (x + ex_of(a) + nx) % nx, yd = (y + ey_of(a) + ny) % ny;
      const size_t j = (size_t)yd * nx + xd;
      double v;
      if (f_in) {
        v = f_in[a * plane + j];
      } else {
        const double r = rho[j], u = ux ? ux[j] : 0.0, w = uy ? uy[j] : 0.0;
        const double eu = ex_of(a) * u + ey_of(a) * w;
        v = w_of<double>(a) * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * (u * u + w * w));
      }
      fs[a] = v;
      rsum += v;
    }
    if constexpr (S::kDev) {
      const float rs = float(rsum);
      float resid = rs;
#pragma unroll
      for (int a = 0; a < kQ; ++a) {
        const typename S::T d = S::from_c(float(fs[a] - double(w_of<float>(a)) * double(rs)));
        dst[a * plane + i] = d;
        resid -= S::to_c(d);
      }
      rho_dst[i] = resid;
    } else {
#pragma unroll
      for (int a = 0; a < kQ; ++a) dst[a * plane + i] = typename S::T(fs[a]);
    }
  }
  if (bad) atomicOr(status, kStatusInvalidInit);
}

// f_a(x, t) = f*_a(x - e_a, t-1) as FP64 [9][ny][nx].
template <class S>
__global__ void get_state_kernel(const typename S::T* src, const float* rho_src, int nx,
                                 int ny, size_t plane, double* f_out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = int(i % nx), y = int(i / nx);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const int xs = (x - ex_of(a) + nx) % nx, ys = (y - ey_of(a) + ny) % ny;
      const size_t j = (size_t)ys * nx + xs;
      double v = double(S::to_c(src[a * plane + j]));
      if constexpr (S::kDev) v += double(w_of<float>(a)) * double(rho_src[j]);
      f_out[a * plane + i] = v;
    }
  }
}

// Per-block FP64 partial sums of all populations of a buffer (mass); the
// second pass adds the partials in a fixed order, so the result does not
// depend on scheduling.
constexpr int kReduceThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* smem) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) smem[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < int(blockDim.x >> 5); ++i) s += smem[i];
  return s;
}

template <class S>
__global__ void __launch_bounds__(kReduceThreads)
mass_partial_kernel(const typename S::T* src, const float* rho_src, size_t plane,
                    double* partial) {
  __shared__ double smem[kReduceThreads / 32];
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane;
       i += (size_t)gridDim.x * blockDim.x) {
    double cell = 0.0;
#pragma unroll
    for (int a = 0; a < kQ; ++a) cell += double(S::to_c(src[a * plane + i]));
    if constexpr (S::kDev) cell += double(rho_src[i]);  // sum_a w_a = 1
    acc += cell;
  }
  const double s = block_sum(acc, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

static __global__ void __launch_bounds__(kReduceThreads)
sum_partials_kernel(const double* partial, int n, double* out) {
  __shared__ double smem[kReduceThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  const double s = block_sum(acc, smem);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace lbm
