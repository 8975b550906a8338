"""Host-side logic of the sweep workloads on synthetic inputs (no GPU):
droplet observables and fits, stability ladders, the sigma crossing, the
coexistence read-out and convergence test of the sequential baseline, the
warm start's fallback rules."""
import numpy as np
import pytest

from oracle import theory as th
from paper_1204_4098_gb300 import calibrate, droplets, inputs, lbm, sweep, warmstart


def test_p_eos_matches_oracle_theory():
    eos = th.CarnahanStarling(0.08)
    rho = np.linspace(0.01, 0.45, 37)
    assert np.allclose(droplets.p_eos(rho, 0.08), eos.p(rho), rtol=1e-14, atol=0)


def test_droplet_observables_of_an_eq24_profile():
    """A sharp Eq. 24 droplet has centre/corner densities rho_l/rho_g and an
    equivalent-area radius close to r0; its pressure jump is the EOS one."""
    n, r0, rg, rl, T = 128, 30.0, 0.02, 0.3, 0.08
    rho = inputs.droplet(n, n, rg, rl, r0, W=0.5)
    z = np.zeros_like(rho)
    obs = droplets.observables(rho, z, z, T)
    assert obs["rho_in"] == pytest.approx(rl, rel=1e-12)
    assert obs["rho_out"] == pytest.approx(rg, rel=1e-9)
    assert obs["radius"] == pytest.approx(r0, rel=5e-3)
    assert obs["dp"] == pytest.approx(droplets.p_eos(rl, T) - droplets.p_eos(rg, T))
    assert obs["max_speed"] == 0.0


def test_laplace_fit_recovers_a_linear_law():
    inst = droplets.laplace_instances(n=64, radii=(10, 15, 20, 25), temps=(0.8,), taus=(1.0,),
                                      schemes=((lbm.SC, 0.0),))
    gamma, c = 3e-3, 1e-6
    res = [{"status": lbm.RUN_CAPPED, "steps": 10, "rho_in": 0.3, "rho_out": 0.02,
            "radius": d["r0"] * 0.98, "dp": gamma / (d["r0"] * 0.98) + c, "max_speed": 1e-3}
           for d in inst]
    fit = droplets.laplace_fits(inst, res)[(0.8, 1.0, lbm.SC, 0.0)]
    assert fit["surface_tension"] == pytest.approx(gamma, rel=1e-9)
    assert fit["intercept"] == pytest.approx(c, rel=1e-6)
    assert fit["r2"] == pytest.approx(1.0, abs=1e-12)
    res[1] = {"status": lbm.RUN_DIVERGED, "steps": 10}
    assert droplets.laplace_fits(inst, res)[(0.8, 1.0, lbm.SC, 0.0)] is None
    res[1] = dict(res[0], radius=0.0, rho_in=0.02)  # dissolved
    assert droplets.laplace_fits(inst, res)[(0.8, 1.0, lbm.SC, 0.0)] is None


def test_thresholds_take_the_lowest_contiguous_stable_temperature():
    temps = [0.9, 0.8, 0.7, 0.6, 0.5]
    inst = droplets.stability_instances(((lbm.EDM, 0.0),), (0.6,), temps)
    ok = {"status": lbm.RUN_CAPPED, "max_speed": 0.01}
    bad = {"status": lbm.RUN_DIVERGED}
    fast = {"status": lbm.RUN_CAPPED, "max_speed": 0.5}  # over the 0.3 criterion
    res = [ok, ok, bad, ok, ok]  # 0.6 and 0.5 stable again below a failure
    assert droplets.thresholds(inst, res)[(lbm.EDM, 0.0, 0.6)] == 0.8
    res = [ok, ok, ok, fast, ok]
    assert droplets.thresholds(inst, res)[(lbm.EDM, 0.0, 0.6)] == 0.7
    res = [bad] + [ok] * 4
    assert droplets.thresholds(inst, res)[(lbm.EDM, 0.0, 0.6)] is None


def test_sigma_crossing_interpolates_linearly():
    sig = np.array([0.08, 0.09, 0.10, 0.11])
    val = 0.01 + 0.1 * (sig - 0.08)
    target = 0.01 + 0.1 * (0.0975 - 0.08)
    assert calibrate._crossing(sig, val, target) == pytest.approx(0.0975, rel=1e-12)
    val_nan = val.copy()
    val_nan[1] = np.nan
    assert calibrate._crossing(sig, val_nan, target) == pytest.approx(0.0975, rel=1e-12)
    assert calibrate._crossing(sig, val, 1.0) is None


def test_coexistence_readout_and_calm_rule():
    rho = inputs.slab_step(8, 16, 0.02, 0.3)
    g, l = sweep._coexistence(rho)
    assert (g, l) == (0.02, 0.3)
    assert sweep._calm(0.3, 0.3 + 1e-9, 1e-9 * 2)
    assert not sweep._calm(0.3, 0.3 + 1e-6, 1e-9)
    assert sweep._calm(0.3, 0.3 + 1e-6, 1e-9, rel=1e-5)


def test_warm_start_rejects_an_unknown_fallback_rule():
    with pytest.raises(ValueError):
        warmstart.run_warm([], None, fallback="sometimes")


def test_warm_start_fallback_rules():
    """The cold-start fallback of a warm run (prediction error above 1e-2,
    taken after the first window, at convergence, or never; divergence
    always restarts; at most one restart per run)."""
    A, C, D, CAP = lbm.RUN_ACTIVE, lbm.RUN_CONVERGED, lbm.RUN_DIVERGED, lbm.RUN_CAPPED
    pred = (0.300, 0.050)
    good = (0.302, 0.0502)  # within 1 % of the prediction
    bad_l = (0.306, 0.050)  # rho_l 2 % off
    bad_g = (0.300, 0.0506)  # rho_g 1.2 % off

    def f(rule, status, windows, fell, obs):
        return warmstart.needs_fallback(rule, status, windows, fell, obs[0], obs[1], pred[0],
                                        pred[1], 1e-2)

    for rule in warmstart.FALLBACK_RULES:
        assert f(rule, D, 5, False, good)  # divergence restarts whatever the rule
        assert not f(rule, D, 5, True, bad_l)  # but only once
    assert f("first_window", A, 1, False, bad_l) and f("first_window", A, 1, False, bad_g)
    assert not f("first_window", A, 1, False, good)
    assert not f("first_window", A, 2, False, bad_l)  # the check is due after window 1 only
    assert f("first_window", C, 1, False, bad_l)
    assert f("converged", C, 7, False, bad_l) and f("converged", C, 7, False, bad_g)
    assert not f("converged", C, 7, False, good)
    assert not f("converged", A, 1, False, bad_l) and not f("converged", CAP, 9, False, bad_l)
    assert not any(f("diverged", st, w, False, bad_l) for st in (A, C, CAP) for w in (1, 7))
    # trend: due at the third window (with the extrapolated limits passed in)
    assert f("trend", A, 3, False, bad_l) and f("trend", C, 3, False, bad_g)
    assert not f("trend", A, 3, False, good)
    assert not f("trend", A, 1, False, bad_l) and not f("trend", A, 2, False, bad_l)
    assert not f("trend", A, 4, False, bad_l)


def test_extrapolated_limit():
    """The fallback's estimate of a run's limits from its last three windows:
    exact for a geometric approach, the last value for noise."""
    q_inf, r = (0.05, 0.30), 0.6
    hist = [(1000 * k, q_inf[0] * (1 - 0.02 * r ** k), q_inf[1] * (1 + 0.01 * r ** k), k)
            for k in range(1, 4)]
    g, l = warmstart.extrapolated_limit(hist)
    assert g == pytest.approx(q_inf[0], rel=1e-12) and l == pytest.approx(q_inf[1], rel=1e-12)
    noisy = [(1000, 0.05, 0.3, 0), (2000, 0.0501, 0.2999, 1), (3000, 0.0500, 0.3001, 2)]
    assert warmstart.extrapolated_limit(noisy) == (0.0500, 0.3001)
    assert warmstart.extrapolated_limit(noisy[:1]) == (0.05, 0.3)


def test_shard_balances_cells_and_covers_every_instance():
    inst = inputs.sweep_instances(40, seed=7)
    parts = [sweep.shard(inst, 3, r) for r in range(3)]
    assert sorted(i for p in parts for i in p) == list(range(40))
    loads = [sum(inst[i]["nx"] * inst[i]["ny"] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(d["nx"] * d["ny"] for d in inst)


class _StandInLattice:
    """Test double of lbm.Lattice for the host loop of sweep.run_sequential:
    a slab whose bulk densities relax geometrically towards fixed values, and
    that reports divergence when its temperature is marked unstable."""

    def __init__(self, nx, ny, T_over_Tc, precision=None, device=0):
        self.nx, self.ny, self.t = nx, ny, T_over_Tc
        self.k = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def init_density(self, rho):
        self.rho0 = np.array(rho)

    def step(self, n, scheme, tau, sigma=0.0, raise_on_error=True):
        self.k += 1
        return lbm.LBM_E_DIVERGED if self.t < 0.5 and self.k == 3 else lbm.LBM_OK

    def observe(self):
        d = 1e-3 * 0.5 ** (8 * self.k)  # settles below the FP32 floor after a few windows
        return (self.rho0 * (1 + d), None, None)


def test_sequential_runner_host_loop(monkeypatch):
    monkeypatch.setattr(sweep.lbm, "Lattice", _StandInLattice)
    inst = [dict(nx=4, ny=32, T_over_Tc=0.8, tau=1.0, sigma=0.0, scheme=lbm.SC),
            dict(nx=4, ny=32, T_over_Tc=0.45, tau=1.0, sigma=0.0, scheme=lbm.SC)]
    res, wall = sweep.run_sequential(inst, [0.05, 0.02], [0.3, 0.35], [0.0, 0.0], window=1000,
                                     max_steps=20000)
    assert res[0]["status"] == lbm.RUN_CONVERGED and res[0]["steps"] < 20000
    assert res[0]["rho_g"] == pytest.approx(0.05, rel=1e-6)
    assert res[0]["rho_l"] == pytest.approx(0.3, rel=1e-6)
    assert [h[0] for h in res[0]["history"]] == list(range(1000, res[0]["steps"] + 1, 1000))
    assert res[1]["status"] == lbm.RUN_DIVERGED and res[1]["steps"] == 3000
    none, _ = sweep.run_sequential(inst[:1], [0.05], [0.3], [0.0], window=1000,
                                   max_steps=5000, conv=lbm.CONV_NONE)
    assert none[0]["status"] == lbm.RUN_CAPPED and none[0]["steps"] == 5000


class _StandInBatch:
    """Test double of lbm.Batch for the host loop of warmstart.run_warm: each
    instance moves to its true densities in its first window after a
    (re)start and converges in its third; instance 2 diverges in its second
    window after the first start."""
    TRUE = {0: (0.050, 0.300), 1: (0.040, 0.320), 2: (0.030, 0.340)}

    def __init__(self, instances, **kw):
        self.n = len(instances)
        self.win = [0] * self.n
        self.steps = [0] * self.n
        self.starts = [0] * self.n
        self.res = [None] * self.n
        self.ms = 0.0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def init_slabs(self, rho_g, rho_l, width):
        self.starts = [1] * self.n

    def init_density(self, k, rho):
        self.win[k] = 0
        self.starts[k] += 1

    def run(self, windows):
        self.ms += 1.0
        for k in range(self.n):
            if self.res[k] is not None and self.res[k]["status"] != lbm.RUN_ACTIVE \
                    and self.win[k] > 0:
                continue
            self.win[k] += 1
            self.steps[k] += 1000
            g, l = self.TRUE[k]
            if k == 2 and self.starts[k] == 1 and self.win[k] == 2:
                st = lbm.RUN_DIVERGED
            else:
                st = lbm.RUN_CONVERGED if self.win[k] >= 3 else lbm.RUN_ACTIVE
            self.res[k] = dict(status=st, steps=self.steps[k], rho_g=g, rho_l=l)
        return sum(r["status"] == lbm.RUN_ACTIVE for r in self.res)

    def stats(self):
        return dict(gpu_ms=self.ms)

    def result(self, k):
        return dict(self.res[k])

    def results(self):
        return [dict(r) for r in self.res]


class _StandInModel:
    def predict(self, instances):
        # instance 1 predicted 5 % off in rho_l; the others within 1 %
        return (np.array([0.301, 0.336, 0.341]), np.array([0.0502, 0.040, 0.0301]),
                np.array([5.0, 5.0, 5.0]))


def test_warm_start_host_loop(monkeypatch):
    monkeypatch.setattr(warmstart.lbm, "Batch", _StandInBatch)
    monkeypatch.setattr(warmstart.sweep, "cold_start_profiles",
                        lambda inst: (np.array([0.05, 0.04, 0.03]), np.array([0.3, 0.32, 0.34])))
    inst = [dict(nx=4, ny=32, T_over_Tc=0.8, tau=1.0, sigma=0.0, scheme=lbm.SC)] * 3
    res, info = warmstart.run_warm(inst, _StandInModel(), fallback="first_window")
    assert [r["fallback"] for r in res] == [False, True, True]
    assert info["fallbacks"] == 2
    assert all(r["status"] == lbm.RUN_CONVERGED for r in res)
    # the restarted runs keep only the history of the run that gave the answer
    assert [len(r["history"]) for r in res] == [3, 3, 3]
    assert res[1]["steps"] == 4000 and res[2]["steps"] == 5000  # wasted steps are counted
    # default: the prediction is judged at the third window against the
    # extrapolated limits (here the settled values), so instance 1 restarts
    # after three windows
    res_t, info_t = warmstart.run_warm(inst, _StandInModel())
    assert [r["fallback"] for r in res_t] == [False, True, True]
    assert res_t[1]["steps"] == 6000 and res_t[2]["steps"] == 5000
    assert all(r["status"] == lbm.RUN_CONVERGED for r in res_t)
    res_c, info_c = warmstart.run_warm(inst, _StandInModel(), fallback="converged")
    assert [r["fallback"] for r in res_c] == [False, True, True]
    res_d, info_d = warmstart.run_warm(inst, _StandInModel(), fallback="diverged")
    assert [r["fallback"] for r in res_d] == [False, False, True]
