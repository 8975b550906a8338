// Host rules of the single-lattice step launch: the kernel variant a context
// resolves to, and the warp-strip geometry of one wave.  Plain C++ without
// CUDA, so that the CPU tests compile and exercise it on its own.
#pragma once

#include <algorithm>

#include "lbm.h"

namespace lbm {

// Shortest band of the automatic geometry: each band reloads the two rows
// around it, so on lattices above 256^2 cells bands stay at least this tall
// even below one full wave.
constexpr int kMinBandRows = 4;

// Shortest automatic band of an nx x ny lattice.  A small lattice's step is
// one short wave (replayed from a graph in runs of steps), whose length is
// the rows each warp walks through, so there the shortest bands win
// (measured, improved scheme, one column per lane: 64^2 and 128^2 2.69 us
// per step with 1-row bands against 4.1-4.2 with 4-row ones; 256^2 3.83 us
// with 2-row bands against 4.36 with 1 or 4; from 512^2 on the 4-row rule
// is as fast or faster).
inline int min_band_rows(int nx, int ny) {
  const long long cells = (long long)nx * ny;
  return cells <= 128LL * 128 ? 1 : (cells <= 256LL * 256 ? 2 : kMinBandRows);
}

// Variant for an nx x ny lattice of `precision` on a GPU of `sm_count` SMs,
// given the requested one; `step` is false for the observe (moments)
// launches, which the staged kernel does not provide.
//  * STAGED only where the bulk copies' 16-byte rule holds (FP32, nx a
//    multiple of 4, at least 64);
//  * PAIR (two columns per lane) needs even nx; AUTO takes it except in FP64,
//    where its doubled register state spills, and on lattices too small to
//    give its 64-column strips (bands of kMinBandRows rows) a quarter of the
//    resident warps, where twice the strips beat the cheaper cells (measured:
//    256^2 1.33x faster with one column per lane, 512^2 equal, 768^2 and up
//    faster with two);
//  * otherwise REGISTER (one column per lane).
inline int resolve_variant(int requested, int precision, int nx, int ny, int sm_count,
                           bool step) {
  const long long pair_items =
      (long long)((nx + 63) / 64) * ((ny + kMinBandRows - 1) / kMinBandRows);
  const bool small = pair_items * 4 < (long long)sm_count * 20;
  const bool pair_ok = nx % 2 == 0;
  const bool staged_ok = step && precision == LBM_FP32 && nx >= 64 && nx % 4 == 0;
  if (requested == LBM_VARIANT_STAGED && staged_ok) return LBM_VARIANT_STAGED;
  if (((requested == LBM_VARIANT_AUTO && precision != LBM_FP64 && !small) ||
       requested == LBM_VARIANT_PAIR) &&
      pair_ok)
    return LBM_VARIANT_PAIR;
  return LBM_VARIANT_REGISTER;
}

struct StripGeometry {
  int n_strips;   // column strips: 32 columns wide, 64 for PAIR
  int band_rows;  // rows per band
  int n_bands;    // bands of rows
  int grid;       // CTAs of warps_per_cta warps, one warp per strip x band
};

// Strips of 32 columns (64 for PAIR) and as many row bands as fill the
// `resident_warps` warp slots once (one wave: every warp of a band runs at the
// same time as its neighbours), at least min_band_rows rows each; a positive
// band_rows_override fixes the band height instead.
inline StripGeometry strip_geometry(int nx, int ny, int variant, long long resident_warps,
                                    int warps_per_cta, int band_rows_override) {
  StripGeometry g;
  const int strip_w = variant == LBM_VARIANT_PAIR ? 64 : 32;
  g.n_strips = (nx + strip_w - 1) / strip_w;
  if (band_rows_override > 0) {
    g.band_rows = std::min(band_rows_override, ny);
  } else {
    long long n_bands = std::max<long long>(1, resident_warps / g.n_strips);
    n_bands = std::min<long long>(n_bands, std::max(1, ny / min_band_rows(nx, ny)));
    g.band_rows = int((ny + n_bands - 1) / n_bands);
  }
  g.n_bands = (ny + g.band_rows - 1) / g.band_rows;
  const long long warps = (long long)g.n_strips * g.n_bands;
  g.grid = int((warps + warps_per_cta - 1) / warps_per_cta);
  return g;
}

}  // namespace lbm
