"""Parameter sweeps of flat-interface runs: batched engine, sequential plain
runs, and sharding across ranks.

* ``cold_start_profiles`` -- per-instance (rho_g, rho_l) from the Maxwell
  construction (Eq. 7) of the library's host EOS helper, i.e. the cold start.
* ``run_batched`` -- all instances in one lbm_batch (CUDA graphs, autotuned).
* ``run_sequential`` -- one plain lbm_step run per instance, with the same
  convergence rule checked on the host after every window (the baseline the
  batched engine is compared with).
* ``shard`` -- longest-processing-time split of instances over ranks (cost =
  cells); ranks run their shards independently (no data-path collective).
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs, lbm

F32_EPS = 2.0 ** -23


def cold_start_profiles(instances, tc_mode=0):
    """(rho_g, rho_l) of the Maxwell construction at each instance's T."""
    g, l = [], []
    for d in instances:
        rg, rl, _ = lbm.maxwell(lbm.temperature(d["T_over_Tc"], tc_mode))
        g.append(rg)
        l.append(rl)
    return np.array(g), np.array(l)


def run_batched(instances, rho_g, rho_l, width, window=1000, tol=1e-9, max_steps=200000,
                mode=lbm.BATCH_AUTO, rows_per_item=0, device=0, stream=None,
                conv=lbm.CONV_COEX, conv_rel=None, trend_tol=None):
    """Run every instance to convergence in one batch; returns (results, stats,
    wall seconds).  width <= 0 starts from a sharp slab."""
    t0 = time.perf_counter()
    with lbm.Batch(instances, window=window, tol=tol, max_steps=max_steps, mode=mode,
                   rows_per_item=rows_per_item, device=device, stream=stream,
                   conv=conv, conv_rel=conv_rel, trend_tol=trend_tol) as b:
        b.init_slabs(rho_g, rho_l, width)
        b.run()
        res, stats = b.results(), b.stats()
    return res, stats, time.perf_counter() - t0


def run_batch_with_history(batch, max_windows=1 << 30):
    """Run a prepared lbm.Batch one window at a time, recording per instance
    the (steps, rho_g, rho_l) after each window it was active in, and the
    cumulative device time after each window.  Returns (history, times)."""
    n = len(batch)
    hist = [[] for _ in range(n)]
    times = []
    active = set(range(n))
    while active and len(times) < max_windows:
        left = batch.run(1)
        times.append(batch.stats()["gpu_ms"] * 1e-3)
        for k in list(active):
            r = batch.result(k)
            hist[k].append((r["steps"], r["rho_g"], r["rho_l"], len(times) - 1))
            if r["status"] != lbm.RUN_ACTIVE:
                active.discard(k)
        if left == 0:
            break
    return hist, times


def answer_step(history, ref_g, ref_l, rtol=1e-3):
    """First recorded step from which rho_g and rho_l stay within rtol of the
    reference values (None if they never settle there); with the window
    index it was recorded at."""
    ok_from = None
    for steps, g, l, w in history:
        good = abs(g / ref_g - 1) <= rtol and abs(l / ref_l - 1) <= rtol
        if good and ok_from is None:
            ok_from = (steps, w)
        elif not good:
            ok_from = None
    return ok_from


def _coexistence(rho):
    ny = rho.shape[0]
    rows = rho.mean(1)
    lo = ny // 2 - 1 if ny >= 2 else 0
    return 0.5 * (rows[0] + rows[-1]), 0.5 * (rows[lo] + rows[ny // 2])


COEX_REL = 8 * F32_EPS  # the batch engine's default relative floor
TREND_TOL = 1e-4        # the batch engine's default TREND bound


def _calm(new, old, tol, rel=COEX_REL):
    return abs(new - old) < max(tol, rel * abs(new))


TREND_BLOCK = 3                # windows per block of the TREND rule
TREND_HIST = 3 * TREND_BLOCK   # windows it looks at


def trend_remaining(d, d_prev):
    """Estimated distance to the limit from the last two changes of block
    means: a geometric decay (same sign, shrinking: r = d / d_prev) has
    |d| r / (1 - r) left; any other pair is noise of amplitude |d| + |d_prev|."""
    if d * d_prev > 0.0 and abs(d) < abs(d_prev):
        r = d / d_prev
        return abs(d) * r / (1.0 - r)
    return abs(d) + abs(d_prev)


def trend_settled(h, bound):
    """TREND on one quantity's last TREND_HIST window values (oldest first):
    the drift of the means of three blocks of TREND_BLOCK windows, and the
    range of the last two blocks (a standing sound wave's amplitude), both
    within bound."""
    m = [float(np.mean(h[b * TREND_BLOCK:(b + 1) * TREND_BLOCK])) for b in range(3)]
    tail = h[TREND_BLOCK:]
    return max(tail) - min(tail) <= bound and trend_remaining(m[2] - m[1], m[1] - m[0]) <= bound


def window_status(conv, c, prev_c, calm, cell, finite, steps, tol, max_steps, rel=COEX_REL,
                  hist=None, trend_tol=TREND_TOL):
    """The batch engine's rule after one window, for runs checked on the host:
    c and prev_c are (rho_g, rho_l) now and one window earlier (prev_c None
    for the first window after a start, which is never calm); hist holds the
    (rho_g, rho_l) of every window since the last start, c last; calm counts
    consecutive windows in which both changed by less than max(tol, rel
    value); cell says every cell changed by less than its tolerance.  Returns
    (status, calm): DIVERGED (a non-finite density) before CONVERGED (CELL:
    cell; COEX: two calm windows in a row; TREND: from the TREND_HIST-th window
    on, both densities settled within max(tol, trend_tol value); NONE: never)
    before CAPPED (steps reached max_steps) before ACTIVE."""
    calm = calm + 1 if (prev_c is not None and _calm(c[0], prev_c[0], tol, rel)
                        and _calm(c[1], prev_c[1], tol, rel)) else 0
    if conv == lbm.CONV_CELL:
        converged = cell
    elif conv == lbm.CONV_COEX:
        converged = calm >= 2
    elif conv == lbm.CONV_TREND:
        converged = hist is not None and len(hist) >= TREND_HIST and all(
            trend_settled([h[i] for h in hist[-TREND_HIST:]], max(tol, trend_tol * abs(c[i])))
            for i in (0, 1))
    else:
        converged = False
    if not finite:
        return lbm.RUN_DIVERGED, calm
    if converged:
        return lbm.RUN_CONVERGED, calm
    if steps >= max_steps:
        return lbm.RUN_CAPPED, calm
    return lbm.RUN_ACTIVE, calm


def run_sequential(instances, rho_g, rho_l, width, window=1000, tol=1e-9, max_steps=200000,
                   device=0, conv=lbm.CONV_COEX, conv_rel=None, trend_tol=None):
    """Plain runs, one instance after another, through lbm_step; convergence
    is checked on the host with the batch engine's rule (window_status:
    CONV_COEX: rho_g and rho_l each changed by less than max(tol, conv_rel
    value) over two consecutive windows; CONV_CELL: every cell by less than
    max(tol, 8 eps_32 rho) over a window; CONV_TREND: both settled within
    max(tol, trend_tol value) over the last nine windows; CONV_NONE: run to
    max_steps).  A smooth profile (width > 0) starts at rest (zero actual
    velocity), a sharp one at u = 0, as in the batch engine's init_slabs.
    Returns (results, wall seconds)."""
    rel = COEX_REL if conv_rel is None else conv_rel
    ttol = TREND_TOL if trend_tol is None else trend_tol
    out = []
    t0 = time.perf_counter()
    for k, d in enumerate(instances):
        ti = time.perf_counter()
        history = []
        nx, ny = d["nx"], d["ny"]
        if width[k] > 0:
            rho0 = inputs.slab_tanh(nx, ny, rho_g[k], rho_l[k], W=width[k])
        else:
            rho0 = inputs.slab_step(nx, ny, rho_g[k], rho_l[k])
        with lbm.Lattice(nx, ny, d["T_over_Tc"], precision=lbm.FP32, device=device) as lat:
            if width[k] > 0 and d["scheme"] != lbm.NOFORCE:
                lat.init_density_at_rest(rho0)
            else:
                lat.init_density(rho0)
            prev = lat.observe()[0]
            prev_c, hist_c = None, []
            steps, status, calm = 0, lbm.RUN_ACTIVE, 0
            while status == lbm.RUN_ACTIVE:
                st = lat.step(window, d["scheme"], d["tau"], d.get("sigma", 0.0),
                              raise_on_error=False)
                steps += window
                if st == lbm.LBM_E_DIVERGED:
                    status = lbm.RUN_DIVERGED
                    break
                rho = lat.observe()[0]
                c = _coexistence(rho)
                hist_c.append(c)
                cell = np.all(np.abs(rho - prev) < np.maximum(tol, 8 * F32_EPS * np.abs(rho)))
                status, calm = window_status(conv, c, prev_c, calm, cell,
                                             bool(np.all(np.isfinite(rho))), steps, tol,
                                             max_steps, rel, hist_c, ttol)
                prev, prev_c = rho, c
                history.append((steps, c[0], c[1], len(history)))
            g, l = _coexistence(prev) if status != lbm.RUN_DIVERGED else (np.nan, np.nan)
        out.append(dict(status=status, steps=steps, rho_g=g, rho_l=l, history=history,
                        wall=time.perf_counter() - ti))
    return out, time.perf_counter() - t0


def shard(instances, world, rank):
    """Indices of the instances rank `rank` runs: largest first onto the
    least-loaded rank (cost = cells), deterministic for every rank."""
    loads = [0] * world
    owner = {}
    order = sorted(range(len(instances)),
                   key=lambda i: (-instances[i]["nx"] * instances[i]["ny"], i))
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        owner[i] = r
        loads[r] += instances[i]["nx"] * instances[i]["ny"]
    return [i for i in range(len(instances)) if owner[i] == rank]


def gather_results(local_idx, local_results, n_total, world):
    """All ranks' results in instance order (torch.distributed all_gather of
    Python objects; a host-side exchange, not on the data path)."""
    if world == 1:
        out = [None] * n_total
        for i, r in zip(local_idx, local_results):
            out[i] = r
        return out
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, list(zip(local_idx, local_results)))
    out = [None] * n_total
    for part in parts:
        for i, r in part:
            out[i] = r
    return out
