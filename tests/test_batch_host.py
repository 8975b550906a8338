"""The batch engine's host logic without a GPU: the grid of a work-list class
kernel, the longest-processing-time assignment of instances to the CTAs of a
persistent window, the window-level autotuner and the convergence rule applied
after each window (paper_1204_4098_gb300/csrc/lbm_batch_host.h, compiled here
with the host C++ compiler through tests/host_shim.cpp)."""
import ctypes
import heapq

import numpy as np
import pytest

from paper_1204_4098_gb300 import lbm

WL, PERS, COOP = 1, 2, 3  # LBM_BATCH_WORKLIST, _PERSISTENT, _COOPERATIVE


@pytest.fixture(scope="module")
def S(host_shim):
    return host_shim


# --- work-list grid -----------------------------------------------------------

@pytest.mark.parametrize("items,want", [(0, 0), (1, 1), (4, 1), (5, 2), (9, 4), (17, 8),
                                        (2000, 512), (2400, 608), (2432, 608), (10 ** 6, 608)])
def test_worklist_grid(S, items, want):
    # 4 warps per CTA, 608 resident CTAs: one item per warp, rounded up to a
    # power of two, at most one wave
    assert S.shim_worklist_grid(items, 4, 608) == want


# --- longest-processing-time assignment ------------------------------------------

def lpt_reference(cells, grid):
    """The same greedy in Python: largest first (ties by id), each onto the
    least-loaded CTA (ties by CTA index)."""
    n = len(cells)
    G = max(1, min(n, grid))
    order = sorted(range(n), key=lambda i: (-cells[i], i))
    heap = [(0, c) for c in range(G)]
    lists = [[] for _ in range(G)]
    for i in order:
        load, c = heapq.heappop(heap)
        lists[c].append(i)
        heapq.heappush(heap, (load + cells[i], c))
    return lists


def run_lpt(S, cells, grid):
    n = len(cells)
    arr = (ctypes.c_longlong * max(n, 1))(*cells)
    begin = (ctypes.c_int * (grid + 1))()
    lst = (ctypes.c_int * max(n, 1))()
    pos = S.shim_lpt(n, arr, grid, begin, lst)
    return pos, list(begin), list(lst)[:n]


@pytest.mark.parametrize("n,grid,seed", [(37, 8, 1), (512, 304, 2), (3, 8, 3), (1, 1, 4),
                                         (0, 5, 5), (100, 1, 6)])
def test_lpt_assignment(S, n, grid, seed):
    cells = [int(c) for c in np.random.default_rng(seed).integers(32 * 128, 512 * 512, n)]
    pos, begin, lst = run_lpt(S, cells, grid)
    assert pos == n and begin[0] == 0 and begin[grid] == n
    assert all(begin[c] <= begin[c + 1] for c in range(grid))
    assert sorted(lst) == list(range(n))  # every instance exactly once
    got = [lst[begin[c]:begin[c + 1]] for c in range(grid)]
    want = lpt_reference(cells, grid)
    assert got[:len(want)] == want and all(not g for g in got[len(want):])
    if n:
        # Graham's bound for the greedy: makespan <= 4/3 of the optimum, and
        # the optimum is at least the largest instance and the mean load
        loads = [sum(cells[i] for i in g) for g in got]
        bound = max(max(cells), sum(cells) / min(grid, n))
        assert max(loads) <= 4.0 / 3.0 * bound + 1e-9


# --- balanced one-wave schedule ---------------------------------------------------

def run_balanced(S, cols, warps, min_rows):
    flat = [v for c in cols for v in c]
    arr = (ctypes.c_int * max(len(flat), 1))(*flat)
    cap = warps + sum(c[1] for c in cols) + 1
    items = (ctypes.c_int * (4 * cap))()
    begin = (ctypes.c_int * (warps + 1))()
    n = S.shim_balanced(len(cols), arr, warps, min_rows, items, begin)
    it = [tuple(items[4 * k:4 * k + 4]) for k in range(n)]
    return it, list(begin)


@pytest.mark.parametrize("warps,min_rows,seed", [(2432, 8, 1), (2432, 8, 2), (64, 8, 3),
                                                 (2432, 200, 4), (7, 1, 5)])
def test_balanced_schedule_covers_every_row_once_in_equal_pieces(S, warps, min_rows, seed):
    rng = np.random.default_rng(seed)
    cols = [(int(i), int(rng.integers(1, 9)), int(rng.integers(1, 520)))
            for i in rng.permutation(40)[:int(rng.integers(1, 40))]]
    items, begin = run_balanced(S, cols, warps, min_rows)
    total = sum(ns * ny for _, ns, ny in cols)
    used = max(1, min(warps, total // min_rows))
    assert begin[0] == 0 and begin[warps] == len(items)
    assert all(begin[w] <= begin[w + 1] for w in range(warps))
    # every (instance, strip, row) exactly once, in order of the concatenation
    seen = []
    for inst, strip, y0, y1 in items:
        assert 0 <= y0 < y1
        seen += [(inst, strip, y) for y in range(y0, y1)]
    want = [(i, s, y) for i, ns, ny in cols for s in range(ns) for y in range(ny)]
    assert seen == want
    # pieces of equal length to one row; warps past `used` idle
    rows = [sum(y1 - y0 for _, _, y0, y1 in items[begin[w]:begin[w + 1]]) for w in range(warps)]
    assert all(r == 0 for r in rows[used:])
    assert max(rows[:used]) - min(rows[:used]) <= 1
    # a piece is cut into items only at strip ends: every item of a warp but
    # its first starts at row 0, every one but its last ends at the strip's end
    ny = {i: n for i, _, n in cols}
    for w in range(used):
        mine = items[begin[w]:begin[w + 1]]
        assert mine
        assert all(it[2] == 0 for it in mine[1:])
        assert all(it[3] == ny[it[0]] for it in mine[:-1])


def test_balanced_schedule_small_sets(S):
    # 3 strips x 10 rows over 8 warps with >= 8 rows each: 3 pieces of 10
    items, begin = run_balanced(S, [(5, 3, 10)], 8, 8)
    assert items == [(5, 0, 0, 10), (5, 1, 0, 10), (5, 2, 0, 10)]
    assert begin == [0, 1, 2, 3, 3, 3, 3, 3, 3]
    # one piece spanning two instances
    items, begin = run_balanced(S, [(0, 1, 3), (1, 1, 4)], 1, 1)
    assert items == [(0, 0, 0, 3), (1, 0, 0, 4)] and begin == [0, 2]
    # nothing to do
    items, begin = run_balanced(S, [], 4, 8)
    assert items == [] and begin == [0, 0, 0, 0, 0]


# --- window-level autotuner --------------------------------------------------------

CANDS = [(WL, 8), (WL, 16), (WL, 32), (WL, 64), (WL, 128), (PERS, 0),
         (COOP, 16), (COOP, 32), (COOP, 64)]


class Tuner:
    def __init__(self, S, cands=CANDS):
        self.S, self.cands = S, cands
        self.h = S.shim_tuner_new()
        for m, r in cands:
            S.shim_tuner_add(self.h, m, r)

    def choose(self, cells, eligible=None):
        elig = [1 if eligible is None or eligible(c) else 0 for c in self.cands]
        e = (ctypes.c_int * len(elig))(*elig)
        m, r = ctypes.c_int(), ctypes.c_int()
        self.S.shim_tuner_choose(self.h, cells, e, ctypes.byref(m), ctypes.byref(r))
        return m.value, r.value

    def record(self, cand, cost):
        self.S.shim_tuner_record(self.h, cand[0], cand[1], cost)

    @property
    def tuned(self):
        return bool(self.S.shim_tuner_tuned(self.h))

    def run(self, cells, costs, windows, eligible=None):
        """`windows` windows: choose, then record the candidate's cost."""
        seen = []
        for _ in range(windows):
            c = self.choose(cells, eligible)
            seen.append(c)
            self.record(c, costs[c])
        return seen

    def __del__(self):
        self.S.shim_tuner_free(self.h)


COSTS = {(WL, 8): 1.5, (WL, 16): 1.1, (WL, 32): 1.0, (WL, 64): 1.2, (WL, 128): 1.35,
         (PERS, 0): 3.0, (COOP, 16): 1.25, (COOP, 32): 1.4, (COOP, 64): 1.6}


def no_pers(c):
    return c[0] != PERS


def test_first_tuning_times_each_eligible_candidate_then_keeps_the_cheapest(S):
    t = Tuner(S)
    seen = t.run(1000, COSTS, 12, no_pers)
    explored = [c for c in CANDS if c[0] != PERS]
    assert seen[:len(explored)] == explored  # in order, the ineligible one left out
    assert t.tuned and set(seen[len(explored):]) == {(WL, 32)}


def test_retune_after_halving_skips_candidates_over_30_percent_dearer(S):
    t = Tuner(S)
    t.run(1000, COSTS, 9, no_pers)  # 8 timing windows, then the choice
    assert t.tuned
    # half the work left: tune again; WL 8 / 128 and COOP 32 / 64 were over
    # 1.3x the best, so only WL 16, 32, 64 and COOP 16 are timed
    seen = t.run(400, COSTS, 6, no_pers)
    assert seen[:4] == [(WL, 16), (WL, 32), (WL, 64), (COOP, 16)]
    assert seen[4:] == [(WL, 32), (WL, 32)]
    # at the next tuning the left-out ones are timed again, and so are the
    # four of this tuning, all within 30 % of the best
    seen = t.run(150, COSTS, 10, no_pers)
    assert seen[:8] == [c for c in CANDS if c[0] != PERS]
    assert seen[8:] == [(WL, 32), (WL, 32)]


def test_a_candidate_slow_in_one_tuning_sits_out_only_the_next(S):
    costs = dict(COSTS)
    t = Tuner(S)
    t.run(1000, costs, 9, no_pers)
    costs[(WL, 16)] = 1.4  # WL 16 turns slow during the second tuning
    seen = t.run(400, costs, 5, no_pers)
    assert seen == [(WL, 16), (WL, 32), (WL, 64), (COOP, 16), (WL, 32)]
    seen = t.run(150, costs, 8, no_pers)
    assert seen == [(WL, 8), (WL, 32), (WL, 64), (WL, 128), (COOP, 16), (COOP, 32),
                    (COOP, 64), (WL, 32)]


def test_persistent_candidate_is_always_timed_again(S):
    t = Tuner(S)
    t.run(1000, COSTS, 10)  # everything eligible (9 timing windows); PERS at 3x the best
    assert t.tuned
    seen = t.run(400, COSTS, 6)
    assert (PERS, 0) in seen[:5]


def test_retune_when_the_choice_becomes_30_percent_dearer(S):
    t = Tuner(S)
    t.run(1000, COSTS, 8, no_pers)
    c = t.choose(1000, no_pers)
    assert c == (WL, 32) and t.tuned
    t.record(c, 1.29)  # within 30 %: keep it
    assert t.choose(1000, no_pers) == (WL, 32) and t.tuned
    t.record((WL, 32), 1.31)  # over 30 %: the next window starts a tuning
    assert t.choose(1000, no_pers) == (WL, 16) and not t.tuned


def test_all_candidates_left_out_are_timed_again(S):
    cands = [(WL, 32), (WL, 64)]
    costs = {(WL, 32): 1.0, (WL, 64): 2.0}
    t = Tuner(S, cands)
    t.run(1000, costs, 3)
    assert t.tuned
    # tuning again with WL 32 no longer eligible and WL 64 left out as slow:
    # rather than choose nothing, WL 64 is timed
    assert t.choose(100, lambda c: c != (WL, 32)) == (WL, 64)


def test_disabled_mode_is_never_chosen(S):
    t = Tuner(S)
    t.S.shim_tuner_disable(t.h, COOP)
    cheap = dict(COSTS)
    cheap.update({(COOP, 16): 0.1, (COOP, 32): 0.1, (COOP, 64): 0.1})
    seen = t.run(1000, cheap, 10, lambda c: c[0] == WL)
    assert all(c[0] == WL for c in seen) and t.tuned


# --- convergence rule after each window --------------------------------------------
EPS8 = 8 * 2.0 ** -23  # the default relative floor


class Instance:
    """One instance's result and calm counter across windows."""

    def __init__(self, S, conv=lbm.CONV_COEX, tol=1e-9, conv_rel=EPS8, window=1000,
                 max_steps=200000):
        self.S, self.rule = S, (conv, tol, conv_rel, window, max_steps)
        self.r = lbm.lbm_result()
        self.calm = ctypes.c_int(0)
        self.first = True

    def window(self, rho_g, rho_l, max_dev=5.0, finite=True, diverged=False):
        obs = (ctypes.c_double * 6)(rho_g, rho_l, 7.5, 1234.5, 1e-6, max_dev)
        st = self.S.shim_window_verdict(*self.rule, obs, int(finite), int(diverged),
                                        int(self.first), ctypes.byref(self.calm),
                                        ctypes.byref(self.r))
        self.first = False
        return st


def test_coex_needs_two_calm_windows_after_the_first(S):
    inst = Instance(S)
    assert inst.window(0.05, 0.30) == lbm.RUN_ACTIVE  # first window: never calm
    assert inst.window(0.05, 0.30) == lbm.RUN_ACTIVE and inst.calm.value == 1
    assert inst.window(0.05, 0.30) == lbm.RUN_CONVERGED and inst.calm.value == 2
    r = inst.r
    assert r.steps == 3000 and (r.rho_g, r.rho_l, r.width, r.mass) == (0.05, 0.30, 7.5, 1234.5)
    assert r.max_drho == pytest.approx(1e-6)


def test_coex_relative_floor_and_reset(S):
    inst = Instance(S)
    inst.window(0.05, 0.30)
    floor_l = EPS8 * 0.30  # 2.9e-7, above tol = 1e-9
    assert inst.window(0.05, 0.30 + 0.9 * floor_l) == lbm.RUN_ACTIVE and inst.calm.value == 1
    # a change above the floor in either density resets the count
    assert inst.window(0.05, 0.30 + 3.0 * floor_l) == lbm.RUN_ACTIVE and inst.calm.value == 0
    assert inst.window(0.05 + 1e-6, 0.30 + 3.0 * floor_l) == lbm.RUN_ACTIVE
    assert inst.calm.value == 0
    assert inst.window(0.05 + 1e-6, 0.30 + 3.0 * floor_l) == lbm.RUN_ACTIVE
    assert inst.window(0.05 + 1e-6, 0.30 + 3.0 * floor_l) == lbm.RUN_CONVERGED
    # with a larger floor the same change counts as calm
    loose = Instance(S, conv_rel=1e-5)
    loose.window(0.05, 0.30)
    assert loose.window(0.05, 0.30 + 3.0 * floor_l) == lbm.RUN_ACTIVE and loose.calm.value == 1


def test_cell_rule_and_no_rule(S):
    cell = Instance(S, conv=lbm.CONV_CELL)
    assert cell.window(0.05, 0.30, max_dev=1.5) == lbm.RUN_ACTIVE
    assert cell.window(0.05, 0.31, max_dev=0.99) == lbm.RUN_CONVERGED  # every cell in tolerance
    none = Instance(S, conv=lbm.CONV_NONE, max_steps=3000)
    assert [none.window(0.05, 0.30, max_dev=0.0) for _ in range(3)] == [
        lbm.RUN_ACTIVE, lbm.RUN_ACTIVE, lbm.RUN_CAPPED]  # runs to the cap


def test_divergence_outranks_convergence_and_the_cap(S):
    inst = Instance(S, conv=lbm.CONV_CELL, max_steps=1000)
    assert inst.window(0.05, 0.30, max_dev=0.0, diverged=True) == lbm.RUN_DIVERGED
    inst = Instance(S, conv=lbm.CONV_CELL)
    assert inst.window(float("nan"), 0.30, max_dev=0.0, finite=False) == lbm.RUN_DIVERGED


def test_convergence_outranks_the_cap(S):
    inst = Instance(S, max_steps=3000)
    inst.window(0.05, 0.30)
    inst.window(0.05, 0.30)
    assert inst.window(0.05, 0.30) == lbm.RUN_CONVERGED  # reached at the cap itself
    capped = Instance(S, max_steps=2000)
    capped.window(0.05, 0.30)
    assert capped.window(0.05, 0.30) == lbm.RUN_CAPPED


@pytest.mark.parametrize("conv", [lbm.CONV_COEX, lbm.CONV_CELL, lbm.CONV_NONE])
@pytest.mark.parametrize("seed", range(12))
def test_sequential_baseline_applies_the_batch_rule(S, conv, seed):
    """sweep.window_status (the host check of the plain sequential runs the
    batch is compared with) and the batch engine's window_verdict reach the
    same status and calm count window after window."""
    from paper_1204_4098_gb300 import sweep
    rng = np.random.default_rng(seed)
    tol, rel, window, max_steps = 1e-9, EPS8, 1000, 25000
    inst = Instance(S, conv=conv, tol=tol, conv_rel=rel, window=window, max_steps=max_steps)
    g, l = 0.05, 0.30
    prev_c, calm, steps = None, 0, 0
    for _ in range(40):
        # no change, a change under the floor, a change over it
        scale = rng.choice([0.0, 0.3, 5.0], p=[0.15, 0.2, 0.65]) * rel
        g *= 1 + scale * rng.choice([-1, 1])
        l *= 1 + scale * rng.choice([-1, 1])
        max_dev = float(rng.choice([0.5, 2.0], p=[0.1, 0.9]))
        finite = bool(rng.random() > 0.04)
        steps += window
        st_py, calm = sweep.window_status(conv, (g, l), prev_c, calm, max_dev < 1.0, finite,
                                          steps, tol, max_steps, rel)
        st_c = inst.window(g, l, max_dev=max_dev, finite=finite)
        assert (st_py, calm) == (st_c, inst.calm.value)
        prev_c = (g, l)
        if st_py != lbm.RUN_ACTIVE:
            break


# ---- TREND rule ---------------------------------------------------------------

def _trend_run(S, seq, tol=1e-9, trend_tol=1e-4, window=1000, max_steps=10 ** 7):
    """Feed (rho_g, rho_l) pairs window after window; returns the 1-based
    window at which the C++ rule says CONVERGED (None if never)."""
    D = ctypes.c_double
    H = S.shim_trend_hist()
    state = (D * (2 + 2 * H))()
    r = lbm.lbm_result()
    for k, (g, l) in enumerate(seq):
        obs = (D * 6)(g, l, 5.0, 1.0, 0.0, 2.0)
        st = S.shim_window_verdict_trend(tol, trend_tol, window, max_steps, obs, int(k == 0),
                                         state, ctypes.byref(r))
        if st == lbm.RUN_CONVERGED:
            return k + 1
    return None


def test_trend_remaining_cases(S):
    # geometric decay 1e-3 -> 5e-4 (r = 0.5): 5e-4 left
    assert S.shim_trend_remaining(5e-4, 1e-3) == pytest.approx(5e-4)
    assert S.shim_trend_remaining(-9e-4, -1e-3) == pytest.approx(9e-4 * 0.9 / 0.1)
    # sign change (noise, oscillation) and growth: the amplitude
    assert S.shim_trend_remaining(2e-6, -3e-6) == pytest.approx(5e-6)
    assert S.shim_trend_remaining(4e-6, 3e-6) == pytest.approx(7e-6)
    assert S.shim_trend_remaining(0.0, 0.0) == 0.0


def _expected_stop(seq, q_inf, ttol, H=9, B=3):
    """First window at which, for both quantities, the range of the last two
    blocks and the last block mean's true distance to the limit are within
    the bound (what the rule computes exactly for a geometric sequence)."""
    for j in range(H, len(seq) + 1):
        ok = True
        for i in (0, 1):
            h = [x[i] for x in seq[j - H:j]]
            bound = ttol * abs(h[-1])
            m2 = np.mean(h[2 * B:])
            ok &= max(h[B:]) - min(h[B:]) <= bound and abs(m2 - q_inf[i]) <= bound * (1 + 1e-9)
        if ok:
            return j
    return None


@pytest.mark.parametrize("ratio", [0.3, 0.6, 0.8, 0.95])
def test_trend_stops_a_geometric_decay_when_settled(S, ratio):
    """q_k = q_inf (1 + A ratio^k): block means decay geometrically too, so
    the extrapolation is exact and the rule stops exactly when the last
    blocks' range and mean are within trend_tol -- and the value there is
    within trend_tol of the limit."""
    q_inf, A, ttol = (0.02, 0.3), 0.05, 1e-4
    seq = [(q_inf[0] * (1 + A * ratio ** k), q_inf[1] * (1 - A * ratio ** k))
           for k in range(1, 600)]
    k = _trend_run(S, seq, trend_tol=ttol)
    assert k is not None and k >= 9
    assert k == _expected_stop(seq, q_inf, ttol)
    g, l = seq[k - 1]
    assert abs(g / q_inf[0] - 1) <= ttol and abs(l / q_inf[1] - 1) <= ttol


def test_trend_does_not_stop_at_a_turning_point_of_a_sound_wave(S):
    """A slab's standing sound wave sampled once per window (period ~4.5
    windows) decaying over ~15 windows: changes of one sign that shrink
    sharply at a turning point must not pass for a settled decay; the rule
    waits until the oscillation itself is below trend_tol."""
    q_inf, ttol = (0.0244, 0.3397), 1e-4
    amp = lambda k: 0.013 * np.exp(-k / 15.0)
    seq = [(q_inf[0] * (1 + amp(k) * np.cos(2 * np.pi * k / 4.5)),
            q_inf[1] * (1 - 0.3 * amp(k) * np.cos(2 * np.pi * k / 4.5))) for k in range(1, 400)]
    k = _trend_run(S, seq, trend_tol=ttol)
    assert k is not None
    assert amp(k) * 1.05 <= 2 * ttol  # the wave has died down to the bound
    assert abs(seq[k - 1][0] / q_inf[0] - 1) <= 2 * ttol


def test_trend_stops_noise_at_the_ninth_window_and_keeps_a_slow_drift(S):
    rng = np.random.default_rng(3)
    noise = [(0.02 * (1 + 3e-6 * rng.standard_normal()), 0.3 * (1 + 3e-6 * rng.standard_normal()))
             for _ in range(20)]
    assert _trend_run(S, noise) == 9
    # a drift decaying with ratio 0.999 per window: 0.3 % away after 200
    # windows, changes of 3e-6 per window -- a floor on single changes would stop it
    drift = [(0.02 * (1 + 0.01 * 0.999 ** k), 0.3) for k in range(1, 200)]
    assert _trend_run(S, drift) is None


@pytest.mark.parametrize("seed", range(8))
def test_sequential_baseline_applies_the_batch_trend_rule(S, seed):
    """sweep.window_status with CONV_TREND (the sequential runs' host check)
    and the batch engine's rule stop at the same window."""
    from paper_1204_4098_gb300 import sweep
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.3, 0.95)
    P = rng.uniform(3.0, 7.0)
    seq = [(0.02 * (1 + 0.02 * r ** k + 2e-3 * np.exp(-k / 12) * np.cos(2 * np.pi * k / P)
                    + 2e-6 * rng.standard_normal()),
            0.3 * (1 - 0.01 * r ** k + 2e-6 * rng.standard_normal())) for k in range(1, 300)]
    k_c = _trend_run(S, seq)
    k_py, prev_c, hist = None, None, []
    for k, c in enumerate(seq):
        hist.append(c)
        st, _ = sweep.window_status(lbm.CONV_TREND, c, prev_c, 0, False, True, 1000 * (k + 1),
                                    1e-9, 10 ** 7, hist=hist, trend_tol=1e-4)
        if st == lbm.RUN_CONVERGED:
            k_py = k + 1
            break
        prev_c = c
    assert k_py == k_c and k_c is not None
