"""Batched sweep engine (lbm_batch_*) on the GPU: same results as the
single-domain path, convergence and divergence handling, and flat-interface
coexistence against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import theory as th
from paper_1204_4098_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

MIXED = [
    dict(nx=45, ny=37, T_over_Tc=0.9, tau=0.8, sigma=0.0, scheme=lbm.SC),
    dict(nx=64, ny=40, T_over_Tc=0.85, tau=0.7, sigma=0.0, scheme=lbm.EDM),
    dict(nx=33, ny=70, T_over_Tc=0.85, tau=0.9, sigma=0.1, scheme=lbm.IMPROVED),
    dict(nx=100, ny=17, T_over_Tc=0.9, tau=1.2, sigma=0.0, scheme=lbm.EDM_MOD),
    dict(nx=32, ny=32, T_over_Tc=0.95, tau=1.0, sigma=0.0, scheme=lbm.LADD),
    dict(nx=7, ny=129, T_over_Tc=0.9, tau=0.6, sigma=0.0, scheme=lbm.NOFORCE),
    dict(nx=130, ny=23, T_over_Tc=0.85, tau=0.8, sigma=0.1, scheme=lbm.IMPROVED),
    dict(nx=2, ny=11, T_over_Tc=0.9, tau=1.0, sigma=0.0, scheme=lbm.SC),
]


def droplet(d, seed):
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(d["T_over_Tc"])))
    return inputs.droplet(d["nx"], d["ny"], rg, rl, min(d["nx"], d["ny"]) / 4.0, W=4.0) * \
        (1 + 1e-3 * np.random.default_rng(seed).uniform(-1, 1, (d["ny"], d["nx"])))


@pytest.mark.parametrize("mode,rows", [(lbm.BATCH_WORKLIST, 8), (lbm.BATCH_WORKLIST, 64),
                                       (lbm.BATCH_WORKLIST_DYNAMIC, 8),
                                       (lbm.BATCH_WORKLIST_DYNAMIC, 32),
                                       (lbm.BATCH_PERSISTENT, 0), (lbm.BATCH_COOPERATIVE, 16),
                                       (lbm.BATCH_COOPERATIVE, 64), (lbm.BATCH_BALANCED, 0),
                                       (lbm.BATCH_AUTO, 0)])
def test_batch_matches_single_domain_bitwise(mode, rows):
    windows, window = 3, 10
    b = lbm.Batch(MIXED, window=window, tol=0.0, max_steps=10 ** 6, mode=mode,
                  rows_per_item=rows)
    rho0 = [droplet(d, k) for k, d in enumerate(MIXED)]
    for k, r in enumerate(rho0):
        b.init_density(k, r)
    assert b.run(windows) == len(MIXED)
    for k, d in enumerate(MIXED):
        single = lbm.Lattice(d["nx"], d["ny"], d["T_over_Tc"], precision=lbm.FP32)
        single.set_variant(lbm.VARIANT_REGISTER)  # the batch takes two columns per lane
        single.init_density(rho0[k])
        single.step(windows * window, d["scheme"], d["tau"], d["sigma"])
        want = single.observe()[0]
        got = b.density(k)
        assert np.array_equal(got, want), (k, np.max(np.abs(got - want)))
        r = b.result(k)
        assert r["steps"] == windows * window and r["status"] == lbm.RUN_ACTIVE


ODD = [dict(nx=nx, ny=ny, T_over_Tc=0.85, tau=0.8, sigma=0.1, scheme=lbm.IMPROVED)
       for nx, ny in ((63, 40), (127, 19), (3, 33), (1, 21), (65, 30), (5, 9))]


@pytest.mark.parametrize("mode,rows", [(lbm.BATCH_WORKLIST, 8), (lbm.BATCH_WORKLIST_DYNAMIC, 16),
                                       (lbm.BATCH_PERSISTENT, 0), (lbm.BATCH_BALANCED, 0)])
def test_batch_odd_widths_on_the_two_column_body_bitwise(mode, rows):
    """Odd nx >= 3 run on the two-column body with rows padded to nx + 3 and
    columns nx, nx + 1 copying columns 0, 1 (nx = 1 stays on one column per
    lane): the last column in lane 31 of a strip (63, 127), the narrowest
    padded width (3), two strips (65), and 1, bit for bit against the
    single-domain one-column kernel."""
    windows, window = 2, 10
    b = lbm.Batch(ODD, window=window, tol=0.0, max_steps=10 ** 6, mode=mode, rows_per_item=rows)
    rho0 = [droplet(d, 10 + k) for k, d in enumerate(ODD)]
    for k, r in enumerate(rho0):
        b.init_density(k, r)
    assert b.run(windows) == len(ODD)
    for k, d in enumerate(ODD):
        single = lbm.Lattice(d["nx"], d["ny"], d["T_over_Tc"], precision=lbm.FP32)
        single.set_variant(lbm.VARIANT_REGISTER)
        single.init_density(rho0[k])
        single.step(windows * window, d["scheme"], d["tau"], d["sigma"])
        assert np.array_equal(b.density(k), single.observe()[0]), d
        got = b.moments(k)
        for g, w in zip(got, single.observe()):
            assert np.array_equal(g, w), d


def test_batch_init_slabs_profile():
    inst = [dict(nx=40, ny=64, T_over_Tc=0.8, tau=1.0, sigma=0.0, scheme=lbm.SC),
            dict(nx=33, ny=50, T_over_Tc=0.9, tau=1.0, sigma=0.0, scheme=lbm.SC)]
    b = lbm.Batch(inst, window=2)
    g = [0.03, 0.05]
    l = [0.3, 0.25]
    b.init_slabs(g, l, [5.0, 0.0])
    want0 = inputs.slab_tanh(40, 64, 0.03, 0.3, W=5.0)
    want1 = inputs.slab_step(33, 50, 0.05, 0.25)
    assert np.allclose(b.density(0), want0, rtol=2e-7)
    assert np.allclose(b.density(1), want1, rtol=2e-7)


def test_batch_divergence_cap_and_convergence():
    """One unstable instance (Shan-Chen, tau = 0.6 at T = 0.45 Tc diverges in a
    few steps), one that cannot converge within the cap, and stable ones."""
    inst = [dict(nx=32, ny=64, T_over_Tc=0.45, tau=0.6, sigma=0.0, scheme=lbm.SC),
            dict(nx=32, ny=64, T_over_Tc=0.9, tau=1.0, sigma=0.0, scheme=lbm.SC),
            dict(nx=48, ny=96, T_over_Tc=0.85, tau=0.8, sigma=0.105, scheme=lbm.IMPROVED)]
    b = lbm.Batch(inst, window=1000, tol=1e-9, max_steps=60000)
    rg, rl = [], []
    for d in inst:
        g_, l_, _ = lbm.maxwell(lbm.temperature(d["T_over_Tc"]))
        rg.append(g_)
        rl.append(l_)
    b.init_slabs(rg, rl, [5.0] * 3)
    assert b.run() == 0
    res = b.results()
    print("batch results:", res)
    assert res[0]["status"] == lbm.RUN_DIVERGED and res[0]["steps"] == 1000
    assert res[1]["status"] == lbm.RUN_CONVERGED
    assert res[2]["status"] == lbm.RUN_CONVERGED
    # the per-cell rule also settles this one (the Shan-Chen slab at 0.9 Tc)
    cell = lbm.Batch(inst[1:2], window=1000, tol=1e-9, max_steps=60000, conv=lbm.CONV_CELL)
    cell.init_slabs(rg[1:2], rl[1:2], [5.0])
    assert cell.run() == 0 and cell.result(0)["status"] == lbm.RUN_CONVERGED
    capped = lbm.Batch(inst[1:2], window=100, tol=0.0, max_steps=300)
    capped.init_slabs(rg[1:2], rl[1:2], [5.0])
    assert capped.run() == 0
    r = capped.result(0)
    assert r["status"] == lbm.RUN_CAPPED and r["steps"] == 300


def test_batch_coexistence_matches_oracle():
    """Converged flat interfaces: FP32 batch vs the FP64 oracle on the same
    slab (x-invariant, so the oracle runs a 2-column copy) after the same
    number of steps."""
    inst = [dict(nx=32, ny=64, T_over_Tc=t, tau=tau, sigma=s, scheme=sch)
            for t, tau, s, sch in ((0.8, 0.8, 0.105, lbm.IMPROVED), (0.9, 1.0, 0.0, lbm.SC),
                                   (0.85, 0.7, 0.0, lbm.EDM), (0.75, 1.0, 0.125, lbm.IMPROVED))]
    b = lbm.Batch(inst, window=1000, tol=1e-9, max_steps=100000)
    mx = [th.maxwell(th.CarnahanStarling(th.temperature(d["T_over_Tc"])))[:2] for d in inst]
    b.init_slabs([m[0] for m in mx], [m[1] for m in mx], [5.0] * len(inst))
    assert b.run() == 0
    for k, d in enumerate(inst):
        r = b.result(k)
        assert r["status"] == lbm.RUN_CONVERGED, r
        ref = oracle.Lattice(2, 64, d["T_over_Tc"])
        ref.init_density(inputs.slab_tanh(2, 64, *mx[k], W=5.0))
        assert ref.step(r["steps"], d["scheme"], d["tau"], d["sigma"])[0] == 0
        rho = ref.observe()[0]
        og = 0.5 * (rho[0].mean() + rho[-1].mean())
        ol = 0.5 * (rho[31].mean() + rho[32].mean())
        assert r["rho_g"] == pytest.approx(og, rel=1e-4), (k, r, og)
        assert r["rho_l"] == pytest.approx(ol, rel=1e-5), (k, r, ol)
        # FP32 repeats the same roundings every step in a steady state, so the
        # mass drifts linearly: measured up to ~4e-9 relative per step
        assert r["mass"] == pytest.approx(64 * 32 * rho.mean(), rel=5e-9 * r["steps"])
