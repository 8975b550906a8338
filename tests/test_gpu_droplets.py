"""Droplet workloads on the batch engine (Sec. III C, Eq. 24): observables
against the FP64 oracle, Laplace's law, and the stability thresholds of
Figs. 1, 2 and 7."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import theory as th
from paper_1204_4098_gb300 import droplets, inputs, lbm

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def oracle_observables(rho, eos):
    """Centre and corner densities, equivalent-area radius and pressure jump
    of a droplet field, written out from their definitions."""
    ny, nx = rho.shape
    r_in, r_out = rho[ny // 2, nx // 2], rho[0, 0]
    radius = np.sqrt((rho - r_out).sum() / (r_in - r_out) / np.pi)
    return r_in, r_out, radius, eos.p(r_in) - eos.p(r_out)


DROPLET_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "droplets_256_oracle.json")


def test_config2_droplets_match_stored_oracle_runs():
    """Config 2 at its own size (256 x 256, Eq. 24 droplet r0 = 30, W = 5,
    T = 0.8 Tc, 2e4 steps, u = 0) against the FP64 oracle's runs stored by
    tests/golden/make_droplet_golden.py: Shan-Chen and the improved scheme
    (sigma = 0.1) at tau = 1, EDM and the improved scheme at sigma = 0.105
    at tau = 0.6, all in one batch from the same initial densities.  Gate:
    centre and corner densities and the equivalent-area radius within 1e-4
    relative (the FP32 density bound); the pressure jump (Eq. 23) within
    what those density errors allow, |p'(rho_in)| 1e-4 rho_in +
    |p'(rho_out)| 1e-4 rho_out."""
    with open(DROPLET_GOLDEN) as f:
        gold = json.load(f)
    n, pts = gold["n"], gold["points"]
    inst = [dict(nx=n, ny=n, T_over_Tc=gold["T_over_Tc"], tau=p["tau"], scheme=p["scheme_id"],
                 sigma=p["sigma"], r0=gold["r0"]) for p in pts]
    res, _ = droplets.run(inst, gold["steps"], W=gold["W"],
                          densities=[(gold["rho_g0"], gold["rho_l0"])] * len(inst))
    eos = th.CarnahanStarling(th.temperature(gold["T_over_Tc"]))
    for p, r in zip(pts, res):
        assert r["status"] == lbm.RUN_CAPPED and r["steps"] == gold["steps"], p
        for k in ("rho_in", "rho_out", "radius"):
            assert abs(r[k] / p[k] - 1) <= 1e-4, (p["scheme"], p["tau"], k, r[k], p[k])
        dp_tol = 1e-4 * (abs(eos.dp(p["rho_in"])) * p["rho_in"]
                         + abs(eos.dp(p["rho_out"])) * p["rho_out"])
        assert abs(r["dp"] - p["dp"]) <= dp_tol, (p["scheme"], r["dp"], p["dp"], dp_tol)
        print(p["scheme"], p["tau"], p["sigma"], {k: f"{r[k] / p[k] - 1:.1e}"
                                                  for k in ("rho_in", "rho_out", "radius", "dp")})


@pytest.mark.parametrize("scheme,sigma", [(lbm.IMPROVED, 0.105), (lbm.SC, 0.0)])
def test_droplet_observables_match_oracle(scheme, sigma):
    n, r0, t, tau, steps = 64, 12, 0.8, 0.8, 3000
    inst = [dict(nx=n, ny=n, T_over_Tc=t, tau=tau, scheme=scheme, sigma=sigma, r0=r0)]
    res, _ = droplets.run(inst, steps)
    got = res[0]
    assert got["status"] == lbm.RUN_CAPPED and got["steps"] == steps
    eos = th.CarnahanStarling(th.temperature(t))
    rg, rl, _ = th.maxwell(eos)
    ref = oracle.Lattice(n, n, t)
    ref.init_density(inputs.droplet(n, n, rg, rl, r0, W=5.0))
    assert ref.step(steps, scheme, tau, sigma)[0] == 0
    rho, vx, vy = ref.observe()
    r_in, r_out, radius, dp = oracle_observables(rho, eos)
    assert got["rho_in"] == pytest.approx(r_in, rel=1e-5)
    assert got["rho_out"] == pytest.approx(r_out, rel=1e-4)
    assert got["radius"] == pytest.approx(radius, rel=1e-5)
    assert got["dp"] == pytest.approx(dp, rel=1e-3)
    speed = np.sqrt(np.max(vx * vx + vy * vy))
    assert got["max_speed"] == pytest.approx(speed, rel=1e-2, abs=1e-7)


def test_batch_moments_match_single_domain_observe():
    inst = [dict(nx=66, ny=40, T_over_Tc=0.85, tau=0.8, scheme=lbm.IMPROVED, sigma=0.1, r0=10),
            dict(nx=45, ny=50, T_over_Tc=0.9, tau=0.7, scheme=lbm.EDM, sigma=0.0, r0=12),
            dict(nx=32, ny=32, T_over_Tc=0.9, tau=1.0, scheme=lbm.NOFORCE, sigma=0.0, r0=8)]
    tc = lbm.critical_point()[1]
    with lbm.Batch(inst, window=10, tol=0.0, max_steps=10 ** 6, conv=lbm.CONV_NONE) as b:
        rho0 = []
        for k, d in enumerate(inst):
            rg, rl, _ = lbm.maxwell(d["T_over_Tc"] * tc)
            rho0.append(inputs.droplet(d["nx"], d["ny"], rg, rl, d["r0"], W=4.0))
            b.init_density(k, rho0[-1])
        b.run(2)
        for k, d in enumerate(inst):
            single = lbm.Lattice(d["nx"], d["ny"], d["T_over_Tc"], precision=lbm.FP32)
            single.init_density(rho0[k])
            single.step(20, d["scheme"], d["tau"], d["sigma"])
            for got, want in zip(b.moments(k), single.observe()):
                assert np.array_equal(got, want), k


def test_laplace_law():
    """Pressure jump linear in 1/R with a vanishing intercept (Laplace)."""
    inst = droplets.laplace_instances(n=128, radii=(14, 18, 24, 30), temps=(0.8,), taus=(1.0,),
                                      schemes=((lbm.IMPROVED, 0.1), (lbm.SC, 0.0)))
    res, _ = droplets.run(inst, 10000)
    fits = droplets.laplace_fits(inst, res)
    for key, f in fits.items():
        assert f is not None, key
        print(key, f["surface_tension"], f["intercept"], f["r2"])
        assert f["r2"] > 0.99, (key, f)
        assert f["surface_tension"] > 0
        assert abs(f["intercept"]) < 3 * f["intercept_se"] + 0.05 * f["surface_tension"] / 14
        assert f["max_speed"] < 0.05


STABILITY_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "stability_oracle.json")


def test_stability_verdicts_match_oracle_and_paper():
    """Figs. 1, 2, 7 on the paper's droplet (200 x 200, r0 = 30, Tc = 0.094,
    initial width W = 4, started at rest: zero actual velocity, Table I).
    At the five reduced temperatures around each printed threshold, the
    GPU's verdict (diverged, or max |v| > 0.3 after 1e4 steps) equals the
    FP64 oracle's stored verdict at every point
    (tests/golden/make_stability_golden.py).  The lowest stable point of
    each ladder then equals the printed value for the improved scheme
    (sigma = 0.105, 0.63), Shan-Chen (0.86) and the two EDM forms at
    tau = 0.7 (0.67, 0.57).  For EDM and Guo's scheme at tau = 0.6 the
    lowest stable point is printed, not gated against the paper: there the
    oracle itself (and so the GPU) is stable one ladder step below the
    printed value, which the paper's unstated budget, width and criterion
    leave open."""
    with open(STABILITY_GOLDEN) as f:
        gold = json.load(f)
    inst, want, dens = [], [], []
    for lad in gold["ladders"]:
        for p in lad["points"]:
            inst.append(dict(nx=gold["n"], ny=gold["n"], T_over_Tc=p["T_over_Tc"],
                             tau=lad["tau"], scheme=lad["scheme_id"], sigma=lad["sigma"],
                             r0=gold["r0"]))
            want.append(p["stable"])
            dens.append((p["rho_g0"], p["rho_l0"]))
    res, info = droplets.run(inst, gold["steps"], W=gold["W"], tc_mode=gold["tc_mode"],
                             at_rest=True, densities=dens)
    got = [not droplets.unstable(r) for r in res]
    mismatch = [(d["scheme"], d["sigma"], d["tau"], d["T_over_Tc"], g, w)
                for d, g, w in zip(inst, got, want) if g != w]
    assert not mismatch, mismatch
    k = 0
    lowest = {}
    for lad in gold["ladders"]:
        pts = lad["points"]  # from the top down
        stable = got[k:k + len(pts)]
        k += len(pts)
        t_min = None
        for p, ok in zip(pts, stable):
            if not ok:
                break
            t_min = p["T_over_Tc"]
        lowest[lad["name"]] = (t_min, lad["printed_lowest_stable"])
    print("lowest stable (GPU = oracle, printed):", lowest, "gpu s", info["gpu_ms"] / 1e3)
    for name in ("IMPROVED_sigma0.105", "SC", "EDM_tau0.7", "EDM_MOD_tau0.7"):
        assert lowest[name][0] == lowest[name][1], (name, lowest[name])
