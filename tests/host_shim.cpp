// C entry points over the host-side rules of the library, compiled by the
// CPU tests with the host C++ compiler (no CUDA) and driven through ctypes:
// the batch engine's scheduling (lbm_batch_host.h) and the single-lattice
// launch rules (lbm_geometry.h).
#include "lbm_batch_host.h"
#include "lbm_geometry.h"

extern "C" {

int shim_worklist_grid(int items, int warps_per_cta, int max_grid) {
  return lbm::worklist_grid(items, warps_per_cta, max_grid);
}

// ids 0..n-1 with costs cells[i]; begin gets grid + 1 entries, list n.
int shim_lpt(int n, const long long* cells, int grid, int* begin, int* list) {
  std::vector<int> ids(n);
  for (int i = 0; i < n; ++i) ids[i] = i;
  int pos = 0;
  lbm::lpt_assign(ids, [cells](int i) { return size_t(cells[i]); }, grid, begin, list, pos);
  return pos;
}

// columns: 3 ints each (instance, strips, rows); items: 4 ints each.
int shim_balanced(int ncols, const int* cols, int warps, int min_rows, int* items, int* begin) {
  std::vector<lbm::BalColumn> c(ncols);
  for (int k = 0; k < ncols; ++k) c[k] = lbm::BalColumn{cols[3 * k], cols[3 * k + 1], cols[3 * k + 2]};
  return lbm::balanced_schedule(c, warps, min_rows, reinterpret_cast<lbm::BalItem*>(items), begin);
}

void* shim_tuner_new() { return new lbm::WindowTuner(); }
void shim_tuner_free(void* t) { delete static_cast<lbm::WindowTuner*>(t); }
void shim_tuner_add(void* t, int mode, int rows) {
  static_cast<lbm::WindowTuner*>(t)->add(mode, rows);
}

// eligible[k] != 0: candidate k may run now.
void shim_tuner_choose(void* t, unsigned long long cells, const int* eligible, int* mode,
                       int* rows) {
  auto* w = static_cast<lbm::WindowTuner*>(t);
  const auto c = w->choose(size_t(cells), [eligible](size_t k) { return eligible[k] != 0; });
  *mode = c.first;
  *rows = c.second;
}

void shim_tuner_record(void* t, int mode, int rows, double cost) {
  static_cast<lbm::WindowTuner*>(t)->record(mode, rows, cost);
}
void shim_tuner_disable(void* t, int mode) {
  static_cast<lbm::WindowTuner*>(t)->disable(mode);
}
int shim_tuner_tuned(void* t) { return static_cast<lbm::WindowTuner*>(t)->tuned ? 1 : 0; }

// One window of the convergence rule: obs = {rho_g, rho_l, width, mass,
// max_abs, max_dev}; r is updated in place; returns the status.
int shim_window_verdict(int conv, double tol, double conv_rel, int window, int max_steps,
                        const double* obs, int finite, int diverged, int first, int* calm,
                        lbm_result* r) {
  lbm::WindowObs o;
  o.rho_g = obs[0];
  o.rho_l = obs[1];
  o.width = obs[2];
  o.mass = obs[3];
  o.max_abs = obs[4];
  o.max_dev = float(obs[5]);
  o.finite = finite != 0;
  o.diverged = diverged != 0;
  const lbm::ConvRule rule{conv, tol, conv_rel, window, max_steps};
  lbm::ConvState st;
  st.calm = *calm;
  st.windows = first ? 0 : 1;
  const int v = lbm::window_verdict(rule, o, first != 0, st, *r);
  *calm = st.calm;
  return v;
}

// The TREND rule with its state carried by the caller in state[2 + 2 H] =
// {calm, windows, hg[H], hl[H]}, H = lbm::kTrendHist; obs as above.
int shim_window_verdict_trend(double tol, double trend_tol, int window, int max_steps,
                              const double* obs, int first, double* state, lbm_result* r) {
  lbm::WindowObs o;
  o.rho_g = obs[0];
  o.rho_l = obs[1];
  o.width = obs[2];
  o.mass = obs[3];
  o.max_abs = obs[4];
  o.max_dev = float(obs[5]);
  o.finite = true;
  o.diverged = false;
  lbm::ConvRule rule{LBM_CONV_TREND, tol, 0.0, window, max_steps};
  rule.trend_tol = trend_tol;
  const int H = lbm::kTrendHist;
  lbm::ConvState st;
  st.calm = int(state[0]);
  st.windows = int(state[1]);
  for (int i = 0; i < H; ++i) {
    st.hg[i] = state[2 + i];
    st.hl[i] = state[2 + H + i];
  }
  const int v = lbm::window_verdict(rule, o, first != 0, st, *r);
  state[0] = st.calm;
  state[1] = st.windows;
  for (int i = 0; i < H; ++i) {
    state[2 + i] = st.hg[i];
    state[2 + H + i] = st.hl[i];
  }
  return v;
}

int shim_trend_hist() { return lbm::kTrendHist; }

double shim_trend_remaining(double d, double d_prev) { return lbm::trend_remaining(d, d_prev); }

int shim_resolve_variant(int requested, int precision, int nx, int ny, int sm_count, int step) {
  return lbm::resolve_variant(requested, precision, nx, ny, sm_count, step != 0);
}

// out = {n_strips, band_rows, n_bands, grid}
void shim_strip_geometry(int nx, int ny, int variant, long long resident_warps,
                         int warps_per_cta, int band_rows_override, int* out) {
  const lbm::StripGeometry g =
      lbm::strip_geometry(nx, ny, variant, resident_warps, warps_per_cta, band_rows_override);
  out[0] = g.n_strips;
  out[1] = g.band_rows;
  out[2] = g.n_bands;
  out[3] = g.grid;
}

int shim_min_band_rows(int nx, int ny) { return lbm::min_band_rows(nx, ny); }

}  // extern "C"
