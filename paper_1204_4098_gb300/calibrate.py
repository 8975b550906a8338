"""Calibration of the improved scheme's sigma against the Maxwell construction.

Sec. IV B fixes sigma numerically: runs with several sigma are compared with
the Maxwell construction and sigma = 0.105 (eps = 16 sigma = 1.68) is found
to fit.  This module automates that search per temperature on the batch
engine: flat-interface slabs (Eq. 36 profile at the Maxwell densities, W = 5,
zero actual velocity) for a grid of sigma at each T/Tc run to convergence (or
to the step cap: at low T the FP32 vapour row means keep moving by a few
ulp, while rho_g has long settled to 1e-5) in one batch; the vapour density
rho_g(sigma) is interpolated linearly where it crosses the Maxwell rho_g,
and a second batch on a finer sigma grid around each crossing refines it.
The result is sigma*(T) and eps*(T) = 16 sigma*.
"""
from __future__ import annotations

import time

import numpy as np

from . import lbm, sweep


def _crossing(sig, val, target):
    """Linear interpolation of the first crossing of val(sig) = target over
    the points with a finite value (runs that failed are skipped)."""
    sig, val = np.asarray(sig, dtype=float), np.asarray(val, dtype=float)
    keep = np.isfinite(val)
    sig, val = sig[keep], val[keep]
    for k in range(len(sig) - 1):
        a, b = val[k] - target, val[k + 1] - target
        if a * b <= 0 and a != b:
            return float(sig[k] + (sig[k + 1] - sig[k]) * a / (a - b))
    return None


def _run(temps, sigmas, tau, nx, ny, max_steps, device):
    inst = [dict(nx=nx, ny=ny, T_over_Tc=float(t), tau=tau, sigma=float(s),
                 scheme=lbm.IMPROVED) for t, ss in zip(temps, sigmas) for s in ss]
    g, l = sweep.cold_start_profiles(inst)
    res, stats, wall = sweep.run_batched(inst, g, l, np.full(len(inst), 5.0),
                                         max_steps=max_steps, device=device)
    out, k = [], 0
    for ss in sigmas:
        rows = res[k:k + len(ss)]
        k += len(ss)
        out.append(np.array([r["rho_g"] if r["status"] in (lbm.RUN_CONVERGED, lbm.RUN_CAPPED)
                             else np.nan for r in rows]))
    return out, stats["gpu_ms"] / 1e3, wall


def sigma_star(temps, sigmas=np.arange(0.07, 0.1451, 0.01), tau=0.8, nx=32, ny=256,
               refine=5, max_steps=200000, device=0):
    """sigma*(T) for each T/Tc in temps.  Returns a list of dicts with the
    Maxwell rho_g, the coarse and fine rho_g(sigma) curves and sigma*, and
    the device time."""
    temps = [float(t) for t in temps]
    tg = [lbm.maxwell(lbm.temperature(t))[0] for t in temps]
    coarse, gpu1, _ = _run(temps, [sigmas] * len(temps), tau, nx, ny, max_steps, device)
    first = [_crossing(sigmas, c, target) for c, target in zip(coarse, tg)]
    gpu2 = 0.0
    fine_s = []
    for s0 in first:
        h = float(sigmas[1] - sigmas[0])
        fine_s.append(np.linspace(s0 - h / 2, s0 + h / 2, refine) if s0 is not None
                      else np.array([]))
    t0 = time.perf_counter()
    fine = [np.array([])] * len(temps)
    todo = [k for k, s in enumerate(fine_s) if len(s)]
    if todo and refine:
        got, gpu2, _ = _run([temps[k] for k in todo], [fine_s[k] for k in todo], tau, nx, ny,
                            max_steps, device)
        for k, v in zip(todo, got):
            fine[k] = v
    out = []
    for k, t in enumerate(temps):
        s_f = _crossing(fine_s[k], fine[k], tg[k]) if len(fine[k]) else None
        best = s_f if s_f is not None else first[k]
        out.append({"T_over_Tc": t, "rho_g_maxwell": tg[k],
                    "sigma_grid": [float(s) for s in sigmas],
                    "rho_g_coarse": [float(v) for v in coarse[k]],
                    "sigma_fine": [float(s) for s in fine_s[k]],
                    "rho_g_fine": [float(v) for v in fine[k]],
                    "sigma_star": best, "eps_star": None if best is None else 16.0 * best})
    return out, {"gpu_s": gpu1 + gpu2, "wall_refine_s": time.perf_counter() - t0}
