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


def test_stability_thresholds():
    """Figs. 1, 2, 7 on the paper's droplet (200 x 200, r0 = 30, Tc = 0.094,
    initial interface width W = 3): the thresholds printed for Shan-Chen
    (0.86), Guo (0.87) and EDM (0.73) at tau = 0.6, and for EDM (0.67) and
    EDM with C_e = 1/tau (0.57) at tau = 0.7, are reproduced to the 0.02
    ladder; the improved scheme (sigma = 0.105, printed 0.63 at tau = 0.6)
    reaches within 0.04 of it, well below EDM."""
    with open(GOLDEN) as f:
        paper = json.load(f)
    p06 = paper["stability_threshold_tau06"]["value"]
    p07 = paper["stability_threshold_modified_edm"]["value"]
    temps = np.round(np.arange(0.91, 0.499, -0.02), 2)
    at06 = ((lbm.IMPROVED, 0.105), (lbm.EDM, 0.0), (lbm.SC, 0.0), (lbm.IMPROVED, 0.0))
    inst = droplets.stability_instances(at06, (0.6,), temps)
    inst += droplets.stability_instances(((lbm.EDM, 0.0), (lbm.EDM_MOD, 0.0)), (0.7,), temps)
    res, info = droplets.run(inst, 10000, W=3.0, tc_mode=1)
    t = droplets.thresholds(inst, res)
    print("thresholds", t, "paper", p06, p07, "gpu s", info["gpu_ms"] / 1e3)
    tol = 0.02 + 1e-9
    assert abs(t[(lbm.SC, 0.0, 0.6)] - p06["SC"]) <= tol
    assert abs(t[(lbm.IMPROVED, 0.0, 0.6)] - p06["GUO"]) <= tol
    assert abs(t[(lbm.EDM, 0.0, 0.6)] - p06["EDM"]) <= tol
    assert abs(t[(lbm.EDM, 0.0, 0.7)] - p07["EDM"]) <= tol
    assert abs(t[(lbm.EDM_MOD, 0.0, 0.7)] - p07["EDM_MOD"]) <= tol
    assert t[(lbm.IMPROVED, 0.105, 0.6)] <= p06["IMPROVED_sigma0.105"] + 0.04 + 1e-9
    assert t[(lbm.IMPROVED, 0.105, 0.6)] < t[(lbm.EDM, 0.0, 0.6)]
