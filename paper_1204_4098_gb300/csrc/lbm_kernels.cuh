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
// strip_run / strip_kernel below is this design with one column per lane;
// strip_run2 / strip2_kernel gives each lane two adjacent columns of a
// 64-column strip (even nx) and, for FP32 and 16-bit storage on single
// lattices, copies the rows it fetches ahead into shared memory with
// per-lane cp.async (two rows in flight, no registers held for them);
// strip_tma_kernel stages the rows in shared memory with bulk copies.  All
// three compute the same values bit for bit.
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
  int nx, ny;                 // ny: rows of the buffers
  int pitch;                  // elements per row of a plane: nx, or nx + 3 for odd nx in the
                              // two-column kernel (columns nx .. nx + 2 copy columns 0 .. 2)
  int y_begin, y_end;         // rows computed (a domain band: the owned rows)
  int out_row0;               // observe mode: output row of buffer row out_row0 is 0
  int n_strips;               // ceil(nx / 32)
  int band_rows;              // rows per warp
  int n_bands;                // ceil((y_end - y_begin) / band_rows)
  size_t plane;               // pitch * ny
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
  const typename S::T d = kCoherent ? __ldcg(A.src + a * A.plane + idx)
                                     : __ldg(A.src + a * A.plane + idx);
  if constexpr (S::kDev) {
    const C r = C(kCoherent ? __ldcg(A.rho_src + idx) : __ldg(A.rho_src + idx));
    return S::decode(mul_rn(w_of<C>(a), r), d);  // w_a rho + d
  } else {
    return S::to_c(d);
  }
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
  const int nx = A.nx, ny = A.ny, pitch = A.pitch;
  const int y0 = A.y_begin + band * A.band_rows;
  const int y1 = min(y0 + A.band_rows, A.y_end);

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
    const int r0 = y * pitch, rm = ym * pitch, rp = yp * pitch;
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
      h = hlane ? pull_one<S, kCoherent>(A, ha, hy * pitch + hsx) : C(0);
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

    const int idx = y * pitch + c;
    const int oidx = (y - A.out_row0) * nx + c;
    if constexpr (MODE == kModeStep) {
      collide<SCHEME>(Pcur, rho0, Fx, Fy, Cz, A.P);
      if (active) {
        if constexpr (S::kDev) {
          // the density plane absorbs the 16-bit rounding of the deviations,
          // so w_a rho_dst + d_a still sums to rho over a (mass conserved)
          C resid = rho0;
#pragma unroll
          for (int a = 0; a < kQ; ++a) {
            const typename S::T d = S::from_c(fma_rn(-w_of<C>(a), rho0, Pcur[a]));
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
        A.out_rho[oidx] = r;
        A.out_vx[oidx] = (double(jx) + 0.5 * double(Fx)) / r;
        A.out_vy[oidx] = (double(jy) + 0.5 * double(Fy)) / r;
      }
    }
    Wm = Wz; Cm = Cz; Em = Ez;
    Wz = Wp; Cz = Cp; Ez = Ep;
    rho0 = rho1;
  };

  C PA[kQ], PB[kQ], PC[kQ];
  C hA = C(0), hB = C(0), hC = C(0);
  // prologue: psi of rows y0 - 1 and y0, populations of y0 (PA) and y0 + 1
  // (PB); the three rows are loaded together (one memory round trip)
  {
    C rdummy;
    load_row(y0 == 0 ? ny - 1 : y0 - 1, PC, hC);
    load_row(y0, PA, hA);
    load_row(y0 + 1 == ny ? 0 : y0 + 1, PB, hB);
    psi_row(PC, hC, Wm, Cm, Em, rdummy);
    psi_row(PA, hA, Wz, Cz, Ez, rho0);
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
// Two columns per lane (even nx, every storage type)
// ---------------------------------------------------------------------------
// The same computation with lane l owning columns x0 + 2l and x0 + 2l + 1 of
// a 64-column strip: populations move as vectors of two (float2, double2,
// bf16x2, half2; deviation storage's density plane as float2), and the
// per-row overhead (indices, halo psi, shuffles, loop control) is shared by
// two cells.  A pull with e_x = +1 takes the left cell's value from
// the previous lane's upper element (shuffle), e_x = -1 the right cell's from
// the next lane's lower element; the strip's two boundary lanes get those
// elements, and the halo densities, from one extra load spread over lanes
// 0-11 (left) and 16-27 (right).  Every per-cell expression is the one of
// strip_run, so results are bit-identical.
template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<__nv_bfloat16> { using type = __nv_bfloat162; };
template <> struct Vec2<__half> { using type = __half2; };

template <bool kCoherent, class V>
__device__ __forceinline__ V load2(const V* p) {
  if constexpr (kCoherent) return __ldcg(p);
  else return __ldg(p);
}

// Asynchronous copies global -> shared (cp.async, completion tracked per
// thread in commit groups): the row fetch of the two-column kernels.  Only
// the wait is a compiler memory barrier: reads of a stage cannot move above
// the wait that completes it, nor below the next wait, which every reuse of
// the stage follows (the prologue places its own barrier where a stage is
// refetched without one).  Issuing and committing copies then does not
// force values held in memory (the batch body's per-item arguments in
// shared memory) to be read again.
template <int N>  // bytes: 4, 8 or 16, both addresses aligned to N
__device__ __forceinline__ void cp_async(void* smem, const void* g) {
  static_assert(N == 4 || N == 8 || N == 16, "cp.async copies 4, 8 or 16 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(
                   unsigned(__cvta_generic_to_shared(smem))),
               "l"(g), "n"(N));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One fetched row of a warp in shared memory, lane-major (each lane writes
// and reads only its own column of every array): the pairs of the 9 planes;
// for deviation storage also the density pair of the row after the pulled
// row (the two before it stay in registers); the lane's extra element (the
// FP32 value, or the aligned 32-bit word holding the 16-bit deviation, plus
// its density).
template <class S>
struct AsyncRow {
  typename Vec2<typename S::T>::type d[kQ][32];
  float2 rr[S::kDev ? 32 : 1];
  unsigned hd[32];
  float hr[S::kDev ? 32 : 1];
};
// Storage whose rows can be fetched asynchronously (FP32 and 16-bit: pairs
// of 4 or 8 bytes; FP64 keeps its rows in registers).
template <class S>
constexpr bool async_fetch() {
  return S::kDev || std::is_same<S, StoreF32>::value;
}
#ifndef LBM_ASYNC_STAGES
#define LBM_ASYNC_STAGES 3
#endif
// stages per warp: kAsyncStages - 1 rows in flight (y + 2, y + 3, ...) while
// row y is computed, plus the stage of row y + 1, already assembled
constexpr int kAsyncStages = LBM_ASYNC_STAGES;

template <class S>
__device__ __forceinline__ AsyncRow<S>* async_rows() {
  __shared__ AsyncRow<S> s_rows[kStripWarpsPerCta * kAsyncStages];
  return s_rows + (threadIdx.x >> 5) * kAsyncStages;
}

// kPadded: rows may have the odd-nx layout (pitch nx + 3, see StripArgs);
// the batch engine's body.  The single-lattice kernels have pitch = nx, even.
// kAsync: fetch rows into shared memory with cp.async where the storage
// allows (async_fetch; non-coherent loads only).  One lattice gains (FP32
// 8192^2 84.5k -> 87.1k, BF16 82.1k -> 87.0k), and so do its short bands
// (2048^2 with 16-row bands: 66.4k -> 73.1k).  The batch body keeps its rows
// in registers: with its item loop and two scheme bodies the row-copy
// variant spills 36-44 B and measured slower (whole default sweep 52.9k
// against 54.6k MLUPS).
template <class S, int SCHEME, int MODE, bool kCoherent = false, bool kPadded = false,
          bool kAsync = true>
__device__ __forceinline__ void strip_run2(const StripArgs<S>& A, int strip, int band,
                                           int lane) {
  using C = typename S::C;
  using T = typename S::T;
  using V = typename Vec2<T>::type;
  using P2 = Pair<C>;  // the lane's two cells (columns ca, ca + 1)
  constexpr bool kNeedPsi = !(MODE == kModeObserveNoForce ||
                              (MODE == kModeStep && SCHEME == kNoForce));
  const unsigned FULL = 0xffffffffu;
  const int nx = A.nx, ny = A.ny, pitch = kPadded ? A.pitch : A.nx;
  // With the rows fetched by cp.async, the buffer pointers and the plane
  // size are held in registers: the batch body's arguments live in shared
  // memory, and reading them there at every row copy measured 10-15 %
  // slower.  On the register-fetch path they stay references to the
  // arguments, which keeps registers free for the held rows.
  constexpr bool kRowCopy = kAsync && async_fetch<S>() && !kCoherent;
  using HoldSrc = std::conditional_t<kRowCopy, const T* const, const T* const&>;
  using HoldDst = std::conditional_t<kRowCopy, T* const, T* const&>;
  using HoldRSrc = std::conditional_t<kRowCopy, const float* const, const float* const&>;
  using HoldRDst = std::conditional_t<kRowCopy, float* const, float* const&>;
  using HoldPlane = std::conditional_t<kRowCopy, const size_t, const size_t&>;
  HoldSrc f_src = A.src;
  HoldDst f_dst = A.dst;
  HoldRSrc r_src = A.rho_src;
  HoldRDst r_dst = A.rho_dst;
  HoldPlane f_plane = A.plane;
  const int y0 = A.y_begin + band * A.band_rows;
  const int y1 = min(y0 + A.band_rows, A.y_end);
  const int x0 = strip * 64;
  const int xa = x0 + 2 * lane;         // left column of this lane
  const bool active_a = xa < nx, active_b = xa + 1 < nx;
  // Even nx (pitch nx): lanes past the edge take the wrapped columns, which
  // serve as the right neighbours.  Odd nx (pitch nx + 3): columns nx .. nx
  // + 2 of every row hold copies of columns 0 .. 2, so the lane whose cell a
  // is the last column nx - 1 has column 0 as its cell b, and the next lane
  // columns 1 and 2 -- the periodic neighbours, with aligned pairs; lanes
  // further out read column 0 (their cells are unused).
  const int ca = (!kPadded || pitch == nx) ? xa % nx : (xa < pitch ? xa : 0);
  // extra-element lanes: 0..8 halo pulls of column x0-1 (plane = lane),
  // 9..11 column x0-1 of planes 1, 5, 8 (e_x = +1), 16..24 halo pulls of
  // column x0+64 (plane = lane-16), 25..27 column x0+64 of planes 3, 6, 7.
  const int q = lane & 15;
  const bool left = lane < 16;
  const int hcol = left ? (x0 - 1 + nx) % nx : (x0 + 64) % nx;
  int qa, qsx;   // plane and source column of this lane's extra element
  bool qlane = true;
  if (q < kQ) {
    qa = q;
    qsx = ((hcol - c_ex[q]) % nx + nx) % nx;
  } else if (q < 12) {
    qa = left ? (q == 9 ? 1 : (q == 10 ? 5 : 8)) : (q == 9 ? 3 : (q == 10 ? 6 : 7));
    qsx = hcol;
  } else {
    qa = 0;
    qsx = 0;
    qlane = false;
  }
  const int qey = c_ey[qa];
  const int hbase = lane & 16;
  bool bad = false;

  // Row y is fetched in two phases: fetch_row issues the loads (raw vectors,
  // this lane's extra element, deviation storage's density pairs) and
  // assemble forms the pulled populations of both cells, which needs the
  // loaded values in shuffles.  The main loop fetches row y + 2 before
  // computing row y and assembles it afterwards, so the loads are in flight
  // during a whole row's arithmetic instead of stalling the shuffles.
  struct Raw {
    V v[kQ];
    C h;
    float2 rr[3];
  };
  // Deviation storage: rows are fetched in sequence (y0 - 1, y0, y0 + 1, ...),
  // and row y needs the density plane of rows y - 1, y, y + 1, so the planes
  // of the last fetch's rows y and y + 1 are kept (ring) and one row is loaded.
  float2 ring0 = make_float2(0.f, 0.f), ring1 = make_float2(0.f, 0.f);
  bool ring_ok = false;
  auto fetch_row = [&](int y, Raw& R) {
    const int ym = y == 0 ? ny - 1 : y - 1;
    const int yp = y == ny - 1 ? 0 : y + 1;
    const int rows[3] = {ym, y, yp};
    {
      int qy = y - qey;
      qy = qy < 0 ? qy + ny : (qy >= ny ? qy - ny : qy);
      R.h = qlane ? pull_one<S, kCoherent>(A, qa, qy * pitch + qsx) : C(0);
    }
    if constexpr (S::kDev) {
      auto plane_row = [&](int r) {
        return load2<kCoherent>(
            reinterpret_cast<const float2*>(r_src + size_t(r) * pitch + ca));
      };
      if (ring_ok) {  // warp-uniform
        R.rr[0] = ring0;
        R.rr[1] = ring1;
      } else {
        R.rr[0] = plane_row(rows[0]);
        R.rr[1] = plane_row(rows[1]);
        ring_ok = true;
      }
      R.rr[2] = plane_row(rows[2]);
      ring0 = R.rr[1];
      ring1 = R.rr[2];
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const int r = rows[1 - ey_of(a)];  // source row y - ey
      R.v[a] =
          load2<kCoherent>(reinterpret_cast<const V*>(f_src + a * f_plane + size_t(r) * pitch + ca));
    }
  };
  // pulled populations of the lane's two cells (P[a].x at ca, .y at ca + 1)
  auto assemble = [&](const Raw& R, P2 (&P)[kQ], C& h) {
    h = R.h;
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const int ex = ex_of(a), ey = ey_of(a);
      P2 v;  // the two values loaded at ca, ca + 1
      if constexpr (S::kDev) {
        v = S::decode2(mul_rn(P2(w_of<C>(a)), P2(R.rr[1 - ey])), R.v[a]);
      } else {
        v = P2(S::to_c(R.v[a].x), S::to_c(R.v[a].y));
      }
      if (ex == 0) {
        P[a] = v;
      } else if (ex == 1) {  // sources x-1: (prev lane's upper, own lower)
        const int k = a == 1 ? 9 : (a == 5 ? 10 : 11);
        const C fromL = __shfl_sync(FULL, h, k);
        const C up = __shfl_up_sync(FULL, v.y(), 1);
        P[a] = P2(lane == 0 ? fromL : up, v.x());
      } else {  // sources x+1: (own upper, next lane's lower)
        const int k = a == 3 ? 25 : (a == 6 ? 26 : 27);
        const C fromR = __shfl_sync(FULL, h, k);
        const C dn = __shfl_down_sync(FULL, v.x(), 1);
        P[a] = P2(v.y(), lane == 31 ? fromR : dn);
      }
    }
  };
  auto load_row = [&](int y, P2 (&P)[kQ], C& h) {
    Raw R;
    fetch_row(y, R);
    assemble(R, P, h);
  };
  auto rho_of = [](const P2 (&P)[kQ]) {
    P2 r = P[0];
#pragma unroll
    for (int a = 1; a < kQ; ++a) r = add_rn(r, P[a]);
    return r;
  };
  // psi of a row around the lane's cells: Cc = (psi(ca), psi(ca + 1)),
  // Wc = (psi(ca - 1), psi(ca)), Ec = (psi(ca + 1), psi(ca + 2))
  auto psi_row = [&](const P2 (&P)[kQ], C h, P2& Wc, P2& Cc, P2& Ec, P2& r) {
    r = rho_of(P);
    if constexpr (kNeedPsi) {
      Cc = psi_of_rho(r, A.P, bad);
      C hr = __shfl_sync(FULL, h, hbase);
#pragma unroll
      for (int a = 1; a < kQ; ++a) hr = add_rn(hr, __shfl_sync(FULL, h, hbase + a));
      const C hp = psi_of_rho(hr, A.P, bad);
      C w = __shfl_up_sync(FULL, Cc.y(), 1);
      C e = __shfl_down_sync(FULL, Cc.x(), 1);
      if (lane == 0) w = hp;
      if (lane == 31) e = hp;
      Wc = P2(w, Cc.x());
      Ec = P2(Cc.y(), e);
    }
  };
  // Eq. 3: F = -G psi(x) sum_a w(|e_a|^2) psi(x + e_a) e_a for both cells
  auto force = [&](P2 Wm, P2 Cm, P2 Em, P2 Wz, P2 Cz, P2 Ez, P2 Wp, P2 Cp, P2 Ep, P2& Fx,
                   P2& Fy) {
    const P2 third = P2(C(1) / C(3)), twelfth = P2(C(1) / C(12));
    const P2 sx = fma_rn(third, sub_rn(Ez, Wz),
                         mul_rn(twelfth, add_rn(sub_rn(Ep, Wp), sub_rn(Em, Wm))));
    const P2 sy = fma_rn(third, sub_rn(Cp, Cm),
                         mul_rn(twelfth, sub_rn(add_rn(Ep, Wp), add_rn(Em, Wm))));
    const P2 gpsi = mul_rn(P2(A.P.minus_G), Cz);
    Fx = mul_rn(gpsi, sx);
    Fy = mul_rn(gpsi, sy);
  };

  P2 P0[kQ], P1[kQ];
  C h1 = C(0);
  // psi ring: rows y-1 (m), y (z)
  P2 Wm = P2(C(0)), Cm = P2(C(0)), Em = P2(C(0)), Wz = P2(C(0)), Cz = P2(C(0)), Ez = P2(C(0));
  P2 r0;
  // Output row y from P0 (its pulled populations) and P1 (row y + 1's);
  // afterwards P0 holds row y + 1 and the psi ring has advanced.
  auto compute_row = [&](int y) {
    P2 Wp = P2(C(0)), Cp = P2(C(0)), Ep = P2(C(0)), r1;
    psi_row(P1, h1, Wp, Cp, Ep, r1);
    P2 Fx = P2(C(0)), Fy = P2(C(0));
    if constexpr (kNeedPsi) force(Wm, Cm, Em, Wz, Cz, Ez, Wp, Cp, Ep, Fx, Fy);
    const size_t idx = size_t(y) * pitch + ca;
    if constexpr (MODE == kModeStep) {
      collide<SCHEME>(P0, r0, Fx, Fy, Cz, A.P);
      if (active_a) {
        // Every active lane stores its two cells as a pair.  With odd nx
        // (pitch nx + 3, columns nx .. nx + 2 holding copies of columns
        // 0 .. 2) the lane whose cell a is the last column has column nx as
        // its cell b; all its inputs (pulls, and psi up to column nx + 1) are
        // copies, so it computes column 0's values exactly and its pair store
        // refreshes that copy.  Lanes 0 and 1 of strip 0 refresh the copies
        // of columns 1 and 2.
        const bool copies = kPadded && pitch != nx && xa < 4;
        const int goff = xa == 0 ? nx + 1 : nx;  // from the lane's pair to its copy
        if constexpr (S::kDev) {
          // the density plane absorbs the 16-bit rounding of the deviations
          P2 res = r0;
#pragma unroll
          for (int a = 0; a < kQ; ++a) {
            const P2 d = fma_rn(P2(-w_of<C>(a)), r0, P0[a]);
            const V v = S::from_c2(d.x(), d.y());
            T* const at = f_dst + a * f_plane + idx;
            *reinterpret_cast<V*>(at) = v;
            if (copies) at[goff] = xa == 0 ? v.y : v.x;
            res = S::sub_from(res, v);
          }
          const float2 rp = make_float2(float(res.x()), float(res.y()));
          *reinterpret_cast<float2*>(r_dst + idx) = rp;
          if (copies) r_dst[idx + goff] = xa == 0 ? rp.y : rp.x;
        } else {
#pragma unroll
          for (int a = 0; a < kQ; ++a) {
            V v;
            v.x = S::from_c(P0[a].x());
            v.y = S::from_c(P0[a].y());
            T* const at = f_dst + a * f_plane + idx;
            *reinterpret_cast<V*>(at) = v;
            if (copies) at[goff] = xa == 0 ? v.y : v.x;
          }
        }
      }
    } else {
      auto out = [&](C p0, C p1, C p2, C p3, C p4, C p5, C p6, C p7, C p8, C rr, C fx, C fy,
                     size_t i) {
        const C jx = (p1 - p3) + (p5 - p6) + (p8 - p7);
        const C jy = (p2 - p4) + (p5 + p6) - (p7 + p8);
        (void)p0;
        const double r = double(rr);
        A.out_rho[i] = r;
        A.out_vx[i] = (double(jx) + 0.5 * double(fx)) / r;
        A.out_vy[i] = (double(jy) + 0.5 * double(fy)) / r;
      };
      const size_t oidx = size_t(y - A.out_row0) * nx + ca;
      if (active_a)
        out(P0[0].x(), P0[1].x(), P0[2].x(), P0[3].x(), P0[4].x(), P0[5].x(), P0[6].x(),
            P0[7].x(), P0[8].x(), r0.x(), Fx.x(), Fy.x(), oidx);
      if (active_b)
        out(P0[0].y(), P0[1].y(), P0[2].y(), P0[3].y(), P0[4].y(), P0[5].y(), P0[6].y(),
            P0[7].y(), P0[8].y(), r0.y(), Fx.y(), Fy.y(), oidx + 1);
    }
    Wm = Wz; Cm = Cz; Em = Ez;
    Wz = Wp; Cz = Cp; Ez = Ep;
    r0 = r1;
#pragma unroll
    for (int a = 0; a < kQ; ++a) P0[a] = P1[a];
  };
  auto wrap = [ny](int y) { return y >= ny ? y - ny : y; };

  if constexpr (kRowCopy) {
    // Rows are copied into shared memory asynchronously (cp.async), so a row
    // in flight holds no registers, and kAsyncStages - 1 rows (y + 2, ...)
    // are in flight while row y is computed.  Each lane waits for its own
    // copies only (cp.async.wait_group) and reads only its own slots.
    AsyncRow<S>* st = async_rows<S>();
    auto fetch_async = [&](int y, AsyncRow<S>& R) {
      const int ym = y == 0 ? ny - 1 : y - 1;
      const int yp = y == ny - 1 ? 0 : y + 1;
      const int rows[3] = {ym, y, yp};
      if (qlane) {
        int qy = y - qey;
        qy = qy < 0 ? qy + ny : (qy >= ny ? qy - ny : qy);
        const size_t e = size_t(qa) * f_plane + size_t(qy) * pitch + qsx;
        if constexpr (S::kDev) {
          cp_async<4>(&R.hd[lane], f_src + (e & ~size_t(1)));  // pitch and plane are even
          cp_async<4>(&R.hr[lane], r_src + size_t(qy) * pitch + qsx);
        } else {
          cp_async<4>(&R.hd[lane], f_src + e);
        }
      }
      if constexpr (S::kDev) {
        if (!ring_ok) {  // the band's first row: the two density rows before it
          ring0 =
              __ldg(reinterpret_cast<const float2*>(r_src + size_t(rows[0]) * pitch + ca));
          ring1 =
              __ldg(reinterpret_cast<const float2*>(r_src + size_t(rows[1]) * pitch + ca));
          ring_ok = true;
        }
        cp_async<8>(&R.rr[lane], r_src + size_t(rows[2]) * pitch + ca);
      }
#pragma unroll
      for (int a = 0; a < kQ; ++a)
        cp_async<sizeof(V)>(&R.d[a][lane],
                            f_src + a * f_plane + size_t(rows[1 - ey_of(a)]) * pitch + ca);
      cp_async_commit();
    };
    auto assemble_async = [&](const AsyncRow<S>& R, P2 (&P)[kQ], C& h) {
      Raw W;
#pragma unroll
      for (int a = 0; a < kQ; ++a) W.v[a] = R.d[a][lane];
      W.h = C(0);
      if constexpr (S::kDev) {
        W.rr[0] = ring0;
        W.rr[1] = ring1;
        W.rr[2] = R.rr[lane];
        ring0 = W.rr[1];
        ring1 = W.rr[2];
        if (qlane) {  // as pull_one: w_a rho + d at the extra element's cell
          const unsigned u = R.hd[lane];
          const unsigned short bits = (qsx & 1) ? (unsigned short)(u >> 16) : (unsigned short)u;
          T t;
          __builtin_memcpy(&t, &bits, sizeof(bits));
          W.h = S::decode(mul_rn(w_of<C>(qa), C(R.hr[lane])), t);
        }
      } else {
        if (qlane) W.h = S::to_c(__uint_as_float(R.hd[lane]));
      }
      assemble(W, P, h);
    };
    // Row r goes to stage (r - y0 + 1) mod kAsyncStages, fetched in order
    // from y0 - 1; every row fetch (or its absence) commits one group, so
    // the groups still pending after row y's fetch are rows y + 2 .. y + D.
    constexpr int D = kAsyncStages - 1;
    {
      P2 rd;
      fetch_async(y0 == 0 ? ny - 1 : y0 - 1, st[0]);
      fetch_async(y0, st[1]);
      fetch_async(wrap(y0 + 1), st[2]);
#pragma unroll
      for (int k = 2; k < D; ++k) {
        if (y0 + k <= y1) fetch_async(wrap(y0 + k), st[k + 1]);
        else cp_async_commit();  // an empty group keeps the count per row
      }
      cp_async_wait<D>();
      assemble_async(st[0], P0, h1);
      psi_row(P0, h1, Wm, Cm, Em, rd);
      asm volatile("" ::: "memory");  // stage 0's reads stay before its refetch
      if (y0 + D <= y1) fetch_async(wrap(y0 + D), st[0]);
      else cp_async_commit();
      cp_async_wait<D>();
      assemble_async(st[1], P0, h1);
      psi_row(P0, h1, Wz, Cz, Ez, r0);
      cp_async_wait<D - 1>();
      assemble_async(st[2], P1, h1);
    }
    int sn = 3 % kAsyncStages, sf = 1;  // stages of rows y + 2 (next) and y + 1 + D
    for (int y = y0; y < y1; ++y) {
      if (y + 1 + D <= y1) fetch_async(wrap(y + 1 + D), st[sf]);  // into row y's stage
      else cp_async_commit();
      compute_row(y);
      if (y + 2 <= y1) {  // warp-uniform
        cp_async_wait<D - 1>();
        assemble_async(st[sn], P1, h1);
      }
      sn = sn == kAsyncStages - 1 ? 0 : sn + 1;
      sf = sf == kAsyncStages - 1 ? 0 : sf + 1;
    }
    cp_async_wait<0>();
  } else {
    Raw next;
    {
      // the three rows before the first are fetched together: one memory
      // round trip at the start of a band instead of three in sequence
      Raw Rm, Rz;
      P2 rd;
      fetch_row(y0 == 0 ? ny - 1 : y0 - 1, Rm);
      fetch_row(y0, Rz);
      fetch_row(wrap(y0 + 1), next);
      assemble(Rm, P0, h1);
      psi_row(P0, h1, Wm, Cm, Em, rd);
      assemble(Rz, P0, h1);
      psi_row(P0, h1, Wz, Cz, Ez, r0);
      assemble(next, P1, h1);
    }
    for (int y = y0; y < y1; ++y) {
      const bool more = y + 2 <= y1;
      if (more) fetch_row(wrap(y + 2), next);
      compute_row(y);
      if (more) assemble(next, P1, h1);  // warp-uniform
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(A.status, kStatusDiverged);
}

#ifndef LBM_STRIP2_MIN_BLOCKS
#define LBM_STRIP2_MIN_BLOCKS 4  // 128 registers: the fetched row and the two assembled rows
#endif
#ifndef LBM_STRIP2_DEV_MIN_BLOCKS
#define LBM_STRIP2_DEV_MIN_BLOCKS 4  // deviation storage (rows in flight in shared memory)
#endif

template <class S, int SCHEME, int MODE>
__global__ void __launch_bounds__(kStripThreads,
                                  S::kDev ? LBM_STRIP2_DEV_MIN_BLOCKS : LBM_STRIP2_MIN_BLOCKS)
strip2_kernel(const StripArgs<S> A) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * kStripThreads + threadIdx.x) >> 5;
  const int strip = gwarp % A.n_strips;  // n_strips counts 64-column strips here
  const int band = gwarp / A.n_strips;
  if (band >= A.n_bands) return;
  strip_run2<S, SCHEME, MODE>(A, strip, band, lane);
}

// ---------------------------------------------------------------------------
// Bulk-copy staged variant (FP32 direct storage, nx % 4 == 0, nx >= 64)
// ---------------------------------------------------------------------------
// The same warp-strip computation, but the rows a warp needs are brought into
// shared memory by the copy engine (cp.async.bulk, completion counted in
// bytes on an mbarrier) up to kTmaStages rows ahead, instead of being held in
// registers: more bytes in flight per SM at fewer registers, and one copy
// instruction per plane-row instead of per-lane address arithmetic.
//
// Stage layout: for each plane a, the 40 floats of source row (r - ey_a) at
// columns x0-4 .. x0+35 (16-byte aligned; covers the pulls of the 32 lanes
// and of both halo columns).  At the domain's left/right edge the periodic
// part comes from a second copy.  Pulled value of lane l, plane a:
// stage[a][4 + l - ex_a]; left halo stage[a][3 - ex_a]; right stage[a][36 - ex_a].
constexpr int kTmaStages = 4;
constexpr int kTmaSpan = 40;
constexpr unsigned kTmaStageBytes = kQ * kTmaSpan * 4;  // 1440
constexpr long long kTmaSpinLimit = 1ll << 20;           // bounded waits

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return unsigned(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(float* dst, const float* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

template <int SCHEME>
__global__ void __launch_bounds__(kStripThreads, 8)
strip_tma_kernel(const StripArgs<StoreF32> A) {
  using C = float;
  __shared__ __align__(128) float s_stage[kStripWarpsPerCta][kTmaStages][kQ][kTmaSpan];
  __shared__ __align__(8) unsigned long long s_bar[kStripWarpsPerCta][kTmaStages];
  constexpr bool kNeedPsi = SCHEME != kNoForce;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gwarp = (blockIdx.x * kStripThreads + threadIdx.x) >> 5;
  const int strip = gwarp % A.n_strips;
  const int band = gwarp / A.n_strips;
  if (band >= A.n_bands) return;  // warp-uniform
  const int nx = A.nx, ny = A.ny;
  const int y0 = A.y_begin + band * A.band_rows;
  const int y1 = min(y0 + A.band_rows, A.y_end);
  const int x0 = strip * 32;
  const bool active = x0 + lane < nx;
  float(*stage)[kQ][kTmaSpan] = s_stage[wib];
  unsigned long long* bar = s_bar[wib];
  if (lane == 0) {
    for (int d = 0; d < kTmaStages; ++d) mbar_init(&bar[d], 1);
    mbar_init_fence();
  }
  __syncwarp();

  // pulled rows r = y0-1 .. y1 (n_rows of them) go through the stages in turn
  const int n_rows = y1 - y0 + 2;
  const int ha = lane & 15;
  const bool hlane = ha < kQ;
  const int hoff = lane < 16 ? 3 - c_ex[ha] : 36 - c_ex[ha];
  const int hbase = lane & 16;
  unsigned phase = 0u;  // bit d: parity to wait for on stage d
  unsigned pending = 0u;
  bool bad = false, timed_out = false;

  auto issue = [&](int k) {  // pulled row y0 - 1 + k into stage k % kTmaStages
    const int d = k % kTmaStages;
    if (lane == 0) mbar_expect_tx(&bar[d], kTmaStageBytes);
    __syncwarp();
    if (lane < kQ) {
      int sr = y0 - 1 + k - c_ey[lane];
      sr = sr < 0 ? sr + ny : (sr >= ny ? sr - ny : sr);
      sr = sr < 0 ? sr + ny : (sr >= ny ? sr - ny : sr);
      const float* row = A.src + size_t(lane) * A.plane + size_t(sr) * nx;
      float* dst = stage[d][lane];
      const int lo = x0 - 4, hi = x0 + 36;
      if (lo < 0) {
        bulk_g2s(dst, row + nx - 4, 16, &bar[d]);
        bulk_g2s(dst + 4, row, 144, &bar[d]);
      } else if (hi > nx) {
        const int n1 = nx - lo;
        bulk_g2s(dst, row + lo, unsigned(n1) * 4u, &bar[d]);
        bulk_g2s(dst + n1, row, unsigned(kTmaSpan - n1) * 4u, &bar[d]);
      } else {
        bulk_g2s(dst, row + lo, kTmaSpan * 4u, &bar[d]);
      }
    }
    pending |= 1u << d;
  };
  auto wait = [&](int k) {
    const int d = k % kTmaStages;
    bool ok = false;
    for (long long it = 0; it < kTmaSpinLimit && !ok; ++it)
      ok = __any_sync(FULL, mbar_try_wait(&bar[d], (phase >> d) & 1u));
    if (ok) {
      phase ^= 1u << d;
      pending &= ~(1u << d);
    }
    return ok;
  };
  auto pulled = [&](int k, C (&P)[kQ], C& h) {
    const int d = k % kTmaStages;
#pragma unroll
    for (int a = 0; a < kQ; ++a) P[a] = stage[d][a][4 + lane - ex_of(a)];
    if constexpr (kNeedPsi) h = hlane ? stage[d][ha][hoff] : C(0);
  };
  auto rho_of = [](const C (&P)[kQ]) {
    C r = P[0];
#pragma unroll
    for (int a = 1; a < kQ; ++a) r = add_rn(r, P[a]);
    return r;
  };
  auto psi_row = [&](const C (&P)[kQ], C h, C& Wv, C& Cv, C& Ev, C& rho_out) {
    rho_out = rho_of(P);
    if constexpr (kNeedPsi) {
      Cv = psi_of_rho(rho_out, A.P, bad);
      C hr = __shfl_sync(FULL, h, hbase);
#pragma unroll
      for (int a = 1; a < kQ; ++a) hr = add_rn(hr, __shfl_sync(FULL, h, hbase + a));
      const C hp = psi_of_rho(hr, A.P, bad);
      Wv = __shfl_up_sync(FULL, Cv, 1);
      Ev = __shfl_down_sync(FULL, Cv, 1);
      if (lane == 0) Wv = hp;
      if (lane == 31) Ev = hp;
    }
  };

  for (int k = 0; k < kTmaStages && k < n_rows; ++k) issue(k);
  C Wm = 0, Cm = 0, Em = 0, Wz = 0, Cz = 0, Ez = 0, rho0 = 0, hdummy = 0, rdummy;
  C Pcur[kQ], Pnext[kQ];
  // prologue: rows y0 - 1 (k = 0) and y0 (k = 1)
  if (!wait(0)) timed_out = true;
  if (!timed_out) {
    pulled(0, Pnext, hdummy);
    psi_row(Pnext, hdummy, Wm, Cm, Em, rdummy);
    __syncwarp();
    if (kTmaStages < n_rows) issue(kTmaStages);
  }
  if (!timed_out && !wait(1)) timed_out = true;
  if (!timed_out) {
    C h;
    pulled(1, Pcur, h);
    psi_row(Pcur, h, Wz, Cz, Ez, rho0);
    __syncwarp();
    if (kTmaStages + 1 < n_rows) issue(kTmaStages + 1);
  }
  for (int y = y0; y < y1 && !timed_out; ++y) {
    const int k = y - y0 + 2;  // pulled row y + 1
    if (!wait(k)) {
      timed_out = true;
      break;
    }
    C h, Wp = 0, Cp = 0, Ep = 0, rho1;
    pulled(k, Pnext, h);
    psi_row(Pnext, h, Wp, Cp, Ep, rho1);
    __syncwarp();
    if (k + kTmaStages < n_rows) issue(k + kTmaStages);

    C Fx = C(0), Fy = C(0);
    if constexpr (kNeedPsi) {
      const C third = C(1) / C(3), twelfth = C(1) / C(12);
      const C sx = fma_rn(third, sub_rn(Ez, Wz),
                          mul_rn(twelfth, add_rn(sub_rn(Ep, Wp), sub_rn(Em, Wm))));
      const C sy = fma_rn(third, sub_rn(Cp, Cm),
                          mul_rn(twelfth, sub_rn(add_rn(Ep, Wp), add_rn(Em, Wm))));
      const C gpsi = mul_rn(A.P.minus_G, Cz);
      Fx = mul_rn(gpsi, sx);
      Fy = mul_rn(gpsi, sy);
    }
    collide<SCHEME>(Pcur, rho0, Fx, Fy, Cz, A.P);
    if (active) {
      const int idx = y * nx + x0 + lane;
#pragma unroll
      for (int a = 0; a < kQ; ++a) A.dst[a * A.plane + idx] = Pcur[a];
    }
    Wm = Wz; Cm = Cz; Em = Ez;
    Wz = Wp; Cz = Cp; Ez = Ep;
    rho0 = rho1;
#pragma unroll
    for (int a = 0; a < kQ; ++a) Pcur[a] = Pnext[a];
  }
  if (timed_out) {
    // drain this warp's copies still in flight (bounded), then report
    for (int d = 0; d < kTmaStages; ++d) {
      if (!((pending >> d) & 1u)) continue;
      for (long long it = 0; it < kTmaSpinLimit; ++it)
        if (__any_sync(FULL, mbar_try_wait(&bar[d], (phase >> d) & 1u))) break;
    }
    if (lane == 0) atomicOr(A.status, kStatusTimeout);
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(A.status, kStatusDiverged);
}

// ---------------------------------------------------------------------------
// initialisation and checkpoint kernels (not on the per-step path)
// ---------------------------------------------------------------------------

// f*_a(x') = f_a(x' + e_a): store a physical state (time t, before the pull)
// so that the next pull reproduces it.  The physical state is either
// f_eq(rho, u) (init) or given populations (set).
// Rows of dst have `pitch` >= nx elements; columns nx .. pitch - 1 (the
// copies of an odd-nx two-column layout) get the state of column
// (x - nx) mod nx.
template <class S>
__global__ void set_state_kernel(typename S::T* dst, float* rho_dst, int nx, int ny, int pitch,
                                 size_t plane, const double* rho, const double* ux,
                                 const double* uy, const double* f_in, Phys<double> P,
                                 unsigned* status) {
  const size_t n = size_t(pitch) * ny;
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int xo = int(i % pitch), y = int(i / pitch);
    const int x = xo < nx ? xo : (xo - nx) % nx;
    if (!f_in && status) (void)psi_of_rho(rho[size_t(y) * nx + x], P, bad);  // domain of psi
    double fs[kQ];
    double rsum = 0.0;
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const int xd = (x + ex_of(a) + nx) % nx, yd = (y + ey_of(a) + ny) % ny;
      const size_t j = (size_t)yd * nx + xd;
      double v;
      if (f_in) {
        v = f_in[a * (size_t(nx) * ny) + j];  // unpadded [9][ny][nx]
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
mass_partial_kernel(const typename S::T* src, const float* rho_src, size_t plane, size_t first,
                    size_t count, double* partial) {
  __shared__ double smem[kReduceThreads / 32];
  double acc = 0.0;
  for (size_t i = first + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < first + count;
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
