// Host-side logic of the batch engine: the grid of a work-list class kernel,
// the longest-processing-time assignment of whole instances to the CTAs of a
// persistent window, the window-level autotuner, and the convergence rule
// applied after each window.  Plain C++ without CUDA, so that the CPU tests
// compile and exercise it on its own.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

#include "lbm.h"

namespace lbm {

// CTAs of a work-list class kernel for `items` strip x band items: enough for
// one item per warp, rounded up to a power of two (so that few distinct window
// graphs arise), at most `max_grid` (one wave of resident CTAs); 0 when there
// is no item.
inline int worklist_grid(int items, int warps_per_cta, int max_grid) {
  if (items <= 0) return 0;
  const int need = (items + warps_per_cta - 1) / warps_per_cta;
  if (need >= max_grid) return max_grid;
  int g = 1;
  while (g < need) g <<= 1;
  return std::min(g, max_grid);
}

// Longest-processing-time assignment of `ids` onto at most `grid` CTAs: the
// largest instance (cost(id), ties by id) first, each onto the least-loaded
// CTA.  CTA c's instances are list[begin[c] .. begin[c + 1]), written from
// position `pos` on (advanced); begin gets grid + 1 entries, and CTAs beyond
// the number of instances get none.
template <class Cost>
void lpt_assign(std::vector<int> ids, const Cost& cost, int grid, int* begin, int* list,
                int& pos) {
  const int G = std::max(1, std::min(int(ids.size()), grid));
  std::sort(ids.begin(), ids.end(), [&](int x, int y) {
    const size_t cx = cost(x), cy = cost(y);
    return cx != cy ? cx > cy : x < y;
  });
  using Load = std::pair<size_t, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int c = 0; c < G; ++c) heap.push({0, c});
  std::vector<std::vector<int>> lists(G);
  for (int i : ids) {
    Load l = heap.top();
    heap.pop();
    lists[l.second].push_back(i);
    heap.push({l.first + cost(i), l.second});
  }
  for (int c = 0; c <= grid; ++c) {
    begin[c] = pos;
    if (c < G && !ids.empty())
      for (int i : lists[c]) list[pos++] = i;
  }
}

// Balanced one-wave schedule of a work-list class.  The rows of every strip
// of the class's instances, laid end to end (instance by instance, strip by
// strip), are cut into `used` pieces of equal row count (to one row), one per
// warp of a resident wave; a piece that crosses from one strip into the next
// becomes one item per strip.  used = min(warps, max(1, total rows /
// min_rows)): pieces stay at least min_rows long, since every item starts
// by fetching the rows on either side of its first one.  Like the
// single-lattice kernel's bands, every warp then does the same work and
// the step ends with all of them, instead of with the last of many small
// items.  Items go to items[] (instance, strip, first row, end row), warp
// w's are items[begin[w] .. begin[w + 1]); begin gets warps + 1 entries.
struct BalItem {
  int inst, strip, y0, y1;
};
struct BalColumn {
  int inst, n_strips, ny;
};
inline int balanced_schedule(const std::vector<BalColumn>& cols, int warps, int min_rows,
                             BalItem* items, int* begin) {
  long long total = 0;
  for (const BalColumn& c : cols) total += (long long)c.n_strips * c.ny;
  const long long used =
      std::max(1LL, std::min<long long>(warps, total / std::max(1, min_rows)));
  int n = 0;
  size_t ci = 0;
  int strip = 0, row = 0;  // the next row not yet assigned
  for (int w = 0; w < warps; ++w) {
    begin[w] = n;
    if (w >= used || ci >= cols.size()) continue;
    // rows [total w / used, total (w + 1) / used) of the concatenation
    long long left = total * (w + 1) / used - total * w / used;
    while (left > 0 && ci < cols.size()) {
      const BalColumn& c = cols[ci];
      const int take = int(std::min<long long>(left, c.ny - row));
      items[n++] = BalItem{c.inst, strip, row, row + take};
      left -= take;
      row += take;
      if (row == c.ny) {
        row = 0;
        if (++strip == c.n_strips) {
          strip = 0;
          ++ci;
        }
      }
    }
  }
  begin[warps] = n;
  return n;
}

// Window-level autotuner.  Each candidate (mode, rows) is timed on one live
// window, the cheapest per cell update is kept, and tuning starts again once
// the active work has halved or the chosen candidate has become 30 % dearer
// per cell update (instances leaving change which band height balances the
// remaining items best).  Every tuning window does live work, but a slow
// candidate wastes part of it: one that was over 30 % dearer than the best at
// the previous tuning is left out of the next one (and timed again at the one
// after); the persistent candidate, which suits the small active sets of a
// sweep's end, is always timed.
struct WindowTuner {
  static constexpr double kSkipped = 1e299;      // left out of this tuning
  static constexpr double kUnavailable = 1e300;  // cannot run on this device

  std::vector<std::pair<int, int>> candidates;  // (mode, rows per item)
  std::vector<double> cost;  // per cell update; < 0: not timed in this tuning
  bool tuned = false;
  size_t tuned_cells = 0;   // active cells when the choice was made
  double tuned_cost = 0.0;  // cost per cell update of the choice
  double last_cost = 0.0;   // of the last window run with it
  std::pair<int, int> cur{LBM_BATCH_WORKLIST, 32};

  void add(int mode, int rows) {
    candidates.push_back({mode, rows});
    cost.push_back(-1.0);
  }

  // (mode, rows) for the next window over `cells` active cells;
  // eligible(k) says whether candidate k may run now.
  std::pair<int, int> choose(size_t cells, const std::function<bool(size_t)>& eligible) {
    if (tuned && (cells * 2 < tuned_cells || last_cost > 1.3 * tuned_cost)) {
      tuned = false;
      double best = 1e300;
      for (double c : cost)
        if (c >= 0 && c < best) best = c;
      for (size_t k = 0; k < cost.size(); ++k) {
        const double c = cost[k];
        const bool slow = c >= 0 && c < kSkipped && c > 1.3 * best &&
                          candidates[k].first != LBM_BATCH_PERSISTENT;
        cost[k] = slow ? kSkipped : -1.0;
      }
    }
    if (!tuned) {
      for (size_t k = 0; k < candidates.size(); ++k)
        if (cost[k] < 0 && eligible(k)) return candidates[k];  // time it next
      double best = 1e300;
      size_t bk = 0;
      for (size_t k = 0; k < candidates.size(); ++k)
        if (cost[k] >= 0 && cost[k] < std::min(best, kSkipped)) {
          best = cost[k];
          bk = k;
        }
      if (best >= kSkipped) {
        // every candidate timed last time was left out: time them again
        bool again = false;
        for (double& c : cost)
          if (c == kSkipped) {
            c = -1.0;
            again = true;
          }
        if (again) return choose(cells, eligible);
      }
      cur = candidates[bk];
      tuned = true;
      tuned_cells = cells;
      tuned_cost = best;
      last_cost = best;
    }
    return cur;
  }

  // The window just run with (mode, rows) cost `c` per cell update; the
  // persistent candidate has no band height.
  void record(int mode, int rows, double c) {
    if (tuned) {
      last_cost = c;
      return;
    }
    for (size_t k = 0; k < candidates.size(); ++k)
      if (candidates[k].first == mode &&
          (mode == LBM_BATCH_PERSISTENT || candidates[k].second == rows) && cost[k] < 0)
        cost[k] = c;
  }

  // Candidates of `mode` cannot run here (e.g. a cooperative launch failed).
  void disable(int mode) {
    for (size_t k = 0; k < candidates.size(); ++k)
      if (candidates[k].first == mode) cost[k] = kUnavailable;
  }
};

// One window's observables of an instance, as the window reduction reports
// them (FP64 row means; the largest density change since the previous window,
// absolute and relative to max(tol, 8 eps rho)).
struct WindowObs {
  double rho_g, rho_l, width, mass;
  double max_abs;  // largest |rho(t) - rho(t - window)|
  float max_dev;   // largest |drho| / max(tol, 8 * 2^-23 * rho)
  bool finite;     // every density finite
  bool diverged;   // the device status flagged divergence
};

struct ConvRule {
  int conv;         // LBM_CONV_COEX, _CELL, _NONE or _TREND
  double tol;       // density-change tolerance per window
  double conv_rel;  // COEX: relative floor
  int window;       // steps per window
  int max_steps;    // step cap
  double trend_tol = 1e-4;  // TREND: relative bound on the distance to the limit
};

// TREND looks at the last kTrendBlock * 3 window values of each coexistence
// density (a flat slab's standing sound wave has a period of a few windows,
// so a single window's change can sit at a turning point of it).
constexpr int kTrendBlock = 3;
constexpr int kTrendHist = 3 * kTrendBlock;

// Per-instance state of the convergence rules, reset by a (re)start.
struct ConvState {
  int calm = 0;       // COEX: consecutive calm windows
  int windows = 0;    // windows since the last (re)start
  double hg[kTrendHist] = {0.0};  // TREND: the last window values of rho_g
  double hl[kTrendHist] = {0.0};  //        and of rho_l (oldest first)
};

// Estimated distance to the limit of a quantity whose last two changes
// (between consecutive block means) were d_prev and d: two changes of the
// same sign, the later smaller, are taken as a geometric decay with ratio
// r = d / d_prev, whose remaining distance is |d| r / (1 - r); anything else
// (a sign change, a growing change) as noise or oscillation of amplitude
// |d| + |d_prev|.
inline double trend_remaining(double d, double d_prev) {
  if (d * d_prev > 0.0 && std::fabs(d) < std::fabs(d_prev)) {
    const double r = d / d_prev;
    return std::fabs(d) * r / (1.0 - r);
  }
  return std::fabs(d) + std::fabs(d_prev);
}

// TREND on one quantity's last kTrendHist window values h (oldest first):
// the block means m0, m1, m2 of three consecutive blocks of kTrendBlock
// windows give the drift's remaining distance trend_remaining(m2 - m1,
// m1 - m0), and the range of the last 2 kTrendBlock values bounds the
// oscillation; both must be within bound.
inline bool trend_settled(const double* h, double bound) {
  double m[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < 3; ++b) {
    for (int i = 0; i < kTrendBlock; ++i) m[b] += h[b * kTrendBlock + i];
    m[b] /= kTrendBlock;
  }
  double lo = h[kTrendBlock], hi = h[kTrendBlock];
  for (int i = kTrendBlock; i < kTrendHist; ++i) {
    lo = std::min(lo, h[i]);
    hi = std::max(hi, h[i]);
  }
  return hi - lo <= bound && trend_remaining(m[2] - m[1], m[1] - m[0]) <= bound;
}

// Apply one window to an instance's result: steps and observables are
// updated, the rule state advanced, and the new status returned: DIVERGED
// (device flag or a non-finite density) before CONVERGED before CAPPED (step
// cap reached) before ACTIVE.  CONVERGED means, by rule: CELL every cell
// within its tolerance; COEX two calm windows in a row, a calm window being
// one in which rho_g and rho_l each changed by less than max(tol, conv_rel
// value) (never the first window after a (re)start); TREND, from the
// kTrendHist-th window after a (re)start on, both coexistence densities
// settled (trend_settled) within max(tol, trend_tol value); NONE never.
inline int window_verdict(const ConvRule& rule, const WindowObs& o, bool first, ConvState& st,
                          lbm_result& r) {
  if (first) st = ConvState{};
  const double dg = first ? 0.0 : o.rho_g - r.rho_g;
  const double dl = first ? 0.0 : o.rho_l - r.rho_l;
  const bool coex_calm =
      !first &&
      std::fabs(dg) < std::max(rule.tol, rule.conv_rel * std::fabs(o.rho_g)) &&
      std::fabs(dl) < std::max(rule.tol, rule.conv_rel * std::fabs(o.rho_l));
  st.calm = coex_calm ? st.calm + 1 : 0;
  for (int i = 0; i + 1 < kTrendHist; ++i) {
    st.hg[i] = st.hg[i + 1];
    st.hl[i] = st.hl[i + 1];
  }
  st.hg[kTrendHist - 1] = o.rho_g;
  st.hl[kTrendHist - 1] = o.rho_l;
  st.windows += 1;
  const bool trend =
      st.windows >= kTrendHist &&
      trend_settled(st.hg, std::max(rule.tol, rule.trend_tol * std::fabs(o.rho_g))) &&
      trend_settled(st.hl, std::max(rule.tol, rule.trend_tol * std::fabs(o.rho_l)));
  r.steps += rule.window;
  r.rho_g = o.rho_g;
  r.rho_l = o.rho_l;
  r.width = o.width;
  r.mass = o.mass;
  r.max_drho = o.max_abs;
  bool converged = false;
  if (rule.conv == LBM_CONV_CELL) converged = o.max_dev < 1.0f;
  else if (rule.conv == LBM_CONV_COEX) converged = st.calm >= 2;
  else if (rule.conv == LBM_CONV_TREND) converged = trend;
  if (o.diverged || !o.finite) return LBM_RUN_DIVERGED;
  if (converged) return LBM_RUN_CONVERGED;
  if (r.steps >= rule.max_steps) return LBM_RUN_CAPPED;
  return LBM_RUN_ACTIVE;
}

}  // namespace lbm
