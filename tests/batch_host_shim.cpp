// C entry points over the batch engine's host scheduling (lbm_batch_host.h),
// compiled by tests/test_batch_host.py with the host C++ compiler (no CUDA) and
// driven through ctypes.
#include "lbm_batch_host.h"

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

}  // extern "C"
