"""Learned warm start of flat-interface sweeps.

A 4 -> 64 -> 64 -> 3 network (lbm_mlp_*, trained on the GPU by the
library's kernels) maps a sweep point (T/Tc, tau, sigma, scheme) to the
relaxed slab's (rho_l, rho_g, interface width W).  New runs then start from
the Eq. 36 profile with the predicted values instead of the Maxwell step
(cold start).  Fallback: a warm run that diverges restarts cold, and so
does one whose prediction error exceeds 1e-2 -- the limits of its rho_l or
rho_g, extrapolated from its first three windows (extrapolated_limit),
differ from the prediction by more than 1e-2 (relative); the steps already
spent are counted.  (The bulk densities themselves are still moved by
~0.5-1 % in the first window while the interface relaxes from the initial
tanh profile, even when the prediction is right to 1e-3, so comparing them
directly restarts good predictions too; run_warm's `fallback` keeps that
rule, the check at convergence and divergence-only for comparison.)  Warm
and cold runs stop by the same batch rule, TREND by default: both
coexistence densities settled to 1e-4 over nine windows (sound-wave range
and extrapolated drift).  Cold runs
remain the reference for the error: the tests and the sweep report compare
warm and cold coexistence densities.

Inputs are scaled to [-1, 1] over the sweep ranges.  The network learns
the answer relative to the Maxwell construction at the same temperature
(computed on the host): targets (rho_l / rho_l^M - 1, log(rho_g / rho_g^M),
log W), standardised with the training set's mean and spread.  rho_g spans
2.5 decades over the sweep's temperatures; the ratio to Maxwell is smooth.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import inputs, lbm, sweep

T_RANGE, TAU_RANGE, SIGMA_RANGE = (0.45, 0.95), (0.6, 1.5), (0.0, 0.2)


def features(instances):
    """(T/Tc, tau, sigma, scheme) scaled to [-1, 1]."""
    def scale(v, lo, hi):
        return 2.0 * (v - lo) / (hi - lo) - 1.0
    return np.array([[scale(d["T_over_Tc"], *T_RANGE), scale(d["tau"], *TAU_RANGE),
                      scale(d.get("sigma", 0.0), *SIGMA_RANGE), float(d["scheme"]) - 1.0]
                     for d in instances], dtype=np.float32)


def glorot_params(seed):
    """Glorot-uniform weights, zero biases, in the lbm_mlp layout."""
    g = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((4, 64), (64, 64), (64, 3)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts += [g.uniform(-lim, lim, fan_in * fan_out), np.zeros(fan_out)]
    return np.concatenate(parts).astype(np.float32)


@dataclass
class WarmStartModel:
    mlp: lbm.MLP
    mean: np.ndarray
    std: np.ndarray
    train_loss: float
    train_seconds: float

    def predict(self, instances):
        """(rho_l, rho_g, W) per instance."""
        y = self.mlp.predict(features(instances)).astype(np.float64) * self.std + self.mean
        mg, ml = sweep.cold_start_profiles(instances)
        return ml * (1.0 + y[:, 0]), mg * np.exp(y[:, 1]), np.exp(y[:, 2])


def targets(instances, rho_l, rho_g, width):
    """Network targets relative to the Maxwell densities at each T."""
    mg, ml = sweep.cold_start_profiles(instances)
    return np.stack([np.asarray(rho_l) / ml - 1.0, np.log(np.asarray(rho_g) / mg),
                     np.log(np.asarray(width))], 1)


def training_data(n_draws, seed=40, ny_range=(128, 512), max_steps=100000, window=1000,
                  conv_rel=None, conv=lbm.CONV_TREND, trend_tol=None):
    """Cold batched runs of narrow (nx = 32) slabs drawn from the sweep
    distribution; the converged ones give (features, targets).  Slabs are
    x-invariant, so the width of the lattice does not change the answer."""
    inst = inputs.sweep_instances(n_draws, seed=seed, nx_range=(32, 32), ny_range=ny_range)
    g, l = sweep.cold_start_profiles(inst)
    res, stats, wall = sweep.run_batched(inst, g, l, np.zeros(len(inst)), window=window,
                                         max_steps=max_steps, conv=conv, conv_rel=conv_rel,
                                         trend_tol=trend_tol)
    keep = [k for k, r in enumerate(res)
            if r["status"] == lbm.RUN_CONVERGED and r["rho_g"] > 0 and r["width"] > 0]
    kept = [inst[k] for k in keep]
    X = features(kept)
    Y = targets(kept, [res[k]["rho_l"] for k in keep], [res[k]["rho_g"] for k in keep],
                [res[k]["width"] for k in keep])
    return X, Y, dict(draws=n_draws, converged=len(keep), gpu_ms=stats["gpu_ms"], wall=wall)


def train(X, Y, stages=((1500, 2e-3), (1500, 5e-4), (1500, 1e-4)), batch=128, seed=0,
          device=0):
    """Adam on the GPU in stages of (epochs, learning rate); each stage is one
    kernel launch, the Adam state carries over between stages."""
    mean, std = Y.mean(0), Y.std(0) + 1e-12
    T = ((Y - mean) / std).astype(np.float32)
    rng = np.random.default_rng(seed)
    mlp = lbm.MLP(glorot_params(seed), device=device)
    t0 = time.perf_counter()
    loss = None
    for epochs, lr in stages:
        order = np.stack([rng.permutation(len(X)) for _ in range(epochs)]).astype(np.int32)
        loss = mlp.train(X, T, order, batch, lr)
    return WarmStartModel(mlp, mean, std, loss, time.perf_counter() - t0)


FALLBACK_RULES = ("trend", "first_window", "converged", "diverged")


def extrapolated_limit(history):
    """(rho_g, rho_l) limits estimated from a run's last three window values
    (history rows (steps, rho_g, rho_l, window)): with d and d_prev the last
    two changes, a geometric decay (same sign, shrinking) ends
    sweep.trend_remaining(d, d_prev) further on in the direction of d; any
    other pair leaves the last value."""
    out = []
    for col in (1, 2):
        q = [h[col] for h in history[-3:]]
        if len(q) < 3:
            out.append(q[-1])
            continue
        d, d_prev = q[2] - q[1], q[1] - q[0]
        if d * d_prev > 0.0 and abs(d) < abs(d_prev):
            out.append(q[2] + np.sign(d) * sweep.trend_remaining(d, d_prev))
        else:
            out.append(q[2])
    return out[0], out[1]


def needs_fallback(rule, status, windows_run, fell, rho_l, rho_g, pred_l, pred_g, tol):
    """Whether a warm run restarts from the cold start after this window.  A
    run falls back at most once (`fell`: it already has), always when it has
    diverged, and otherwise when the prediction-error check of `rule` is due
    and rho_l or rho_g differs from its prediction by more than `tol`
    (relative): at the run's third window, with rho_l, rho_g the limits
    extrapolated from its trend ("trend"; the caller passes them), after its
    first window ("first_window"), when it has converged ("converged"), or
    never ("diverged")."""
    if fell:
        return False
    if status == lbm.RUN_DIVERGED:
        return True
    off = abs(rho_l / pred_l - 1) > tol or abs(rho_g / pred_g - 1) > tol
    due = (rule == "converged" and status == lbm.RUN_CONVERGED) or \
        (rule == "first_window" and windows_run == 1) or \
        (rule == "trend" and (windows_run == 3 or
                              (windows_run < 3 and status == lbm.RUN_CONVERGED)))
    return due and off


def run_warm(instances, model, window=1000, tol=1e-9, max_steps=200000, fallback_tol=1e-2,
             device=0, conv_rel=None, fallback="trend", conv=lbm.CONV_TREND, trend_tol=None):
    """Warm-started batched runs with the cold-start fallback, checked after
    every window.  A warm run that diverges restarts at once from the cold
    start (its steps so far are counted; a run falls back at most once).  The
    prediction-error check (relative difference of rho_l or rho_g from the
    prediction above fallback_tol) is taken, by `fallback`:
      "trend"        -- at the third window, against the limits
                        extrapolated from the run's trend (default: the
                        relaxing interface still moves the bulk densities
                        by ~1 % in the first window, not their limits);
      "first_window" -- after the first window (a restart then wastes one
                        window);
      "converged"    -- when the warm run has converged;
      "diverged"     -- never (divergence only).
    Returns (results, info); results carry per-window histories of the run
    that produced the answer.  Runs stop by the batch rule `conv` (TREND by
    default, the same for the cold runs they are compared with)."""
    if fallback not in FALLBACK_RULES:
        raise ValueError(f"unknown fallback rule {fallback!r}")
    pl, pg, pw = model.predict(instances)
    cg, cl = sweep.cold_start_profiles(instances)
    # the network never saw unstable points; keep its answers in a plausible
    # band around Maxwell (and inside the domain of psi)
    pl = np.clip(pl, 0.9 * cl, 1.1 * cl)
    pg = np.clip(pg, 0.1 * cg, 10.0 * cg)
    pw = np.clip(pw, 1.0, 50.0)
    t0 = time.perf_counter()
    n = len(instances)
    hist = [[] for _ in range(n)]
    times = []
    fell = set()
    with lbm.Batch(instances, window=window, tol=tol, max_steps=max_steps, device=device,
                   conv=conv, conv_rel=conv_rel, trend_tol=trend_tol) as b:
        b.init_slabs(pg, pl, pw)
        active = set(range(n))
        while active:
            b.run(1)
            times.append(b.stats()["gpu_ms"] * 1e-3)
            for k in list(active):
                r = b.result(k)
                hist[k].append((r["steps"], r["rho_g"], r["rho_l"], len(times) - 1))
                el, eg = r["rho_l"], r["rho_g"]
                if fallback == "trend":
                    eg, el = extrapolated_limit(hist[k])
                if needs_fallback(fallback, r["status"], len(hist[k]), k in fell, el, eg,
                                  pl[k], pg[k], fallback_tol):
                    d = instances[k]
                    fell.add(k)
                    hist[k] = []
                    b.init_density(k, inputs.slab_step(d["nx"], d["ny"], cg[k], cl[k]))
                elif r["status"] != lbm.RUN_ACTIVE:
                    active.discard(k)
        res, stats = b.results(), b.stats()
    for k, r in enumerate(res):
        r["fallback"] = k in fell
        r["history"] = hist[k]
    return res, dict(gpu_ms=stats["gpu_ms"], wall=time.perf_counter() - t0,
                     fallbacks=len(fell), predicted=(pl, pg, pw), window_times=times)


def run_cold_batched(instances, window=1000, tol=1e-9, max_steps=200000, device=0,
                     conv_rel=None, conv=lbm.CONV_TREND, trend_tol=None):
    cg, cl = sweep.cold_start_profiles(instances)
    t0 = time.perf_counter()
    with lbm.Batch(instances, window=window, tol=tol, max_steps=max_steps, device=device,
                   conv=conv, conv_rel=conv_rel, trend_tol=trend_tol) as b:
        b.init_slabs(cg, cl, np.zeros(len(instances)))
        hist, times = sweep.run_batch_with_history(b)
        res, stats = b.results(), b.stats()
    for k, r in enumerate(res):
        r["history"] = hist[k]
    return res, dict(gpu_ms=stats["gpu_ms"], wall=time.perf_counter() - t0, window_times=times)


def time_to_answer(res, info, ref, rtol=1e-3, among=None):
    """Device time until every run in `among` (default: those whose reference
    converged) has rho_g and rho_l settled within rtol of the reference (cold
    converged) values -- the batch runs them together, so this is the time of
    the latest such window -- and the mean steps to that point.  A run that
    never settles counts with all its steps."""
    if among is None:
        among = [k for k in range(len(res)) if ref[k]["status"] == lbm.RUN_CONVERGED]
    last_w, steps = -1, []
    for k in among:
        r = res[k]
        a = sweep.answer_step(r["history"], ref[k]["rho_g"], ref[k]["rho_l"], rtol)
        if a is None:
            a = (r["steps"], r["history"][-1][3] if r["history"] else len(info["window_times"]) - 1)
        steps.append(a[0])
        last_w = max(last_w, a[1])
    t = info["window_times"][last_w] if last_w >= 0 else 0.0
    return t, float(np.mean(steps)) if steps else None
