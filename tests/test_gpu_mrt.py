"""The multiple-relaxation-time form of the improved scheme (LBM_SCHEME_MRT,
the extension stated at the end of Sec. IV) on the GPU against the FP64
oracle's MRT collision, and its consistency with the BGK improved scheme."""
import numpy as np
import pytest

import oracle
from oracle import theory as th
from paper_1204_4098_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

RATES = (0.8, 1.1, 1.3)  # s_e, s_eps, s_q


def droplet_state(nx, ny, t, seed=0):
    eos = th.CarnahanStarling(th.temperature(t))
    rg, rl, _ = th.maxwell(eos)
    rho = inputs.droplet(nx, ny, rg, rl, min(nx, ny) / 4.0, W=4.0)
    rng = np.random.default_rng(seed)
    return rho, 0.01 * rng.uniform(-1, 1, (ny, nx)), 0.01 * rng.uniform(-1, 1, (ny, nx))


def run(nx, ny, precision, variant, steps, rates, tau=0.8, sigma=0.1, t=0.9):
    rho, ux, uy = droplet_state(nx, ny, t)
    g = lbm.Lattice(nx, ny, t, precision=precision)
    g.set_variant(variant)
    g.set_mrt_rates(*rates)
    g.init_density(rho, ux, uy)
    g.step(steps, lbm.MRT, tau, sigma)
    return g, (rho, ux, uy)


@pytest.mark.parametrize("precision,tol", [(lbm.FP32, 2e-6), (lbm.FP64, 1e-13)])
@pytest.mark.parametrize("nx,ny,variant", [(45, 37, lbm.VARIANT_REGISTER),
                                           (200, 67, lbm.VARIANT_PAIR)])
def test_mrt_matches_oracle(precision, tol, nx, ny, variant):
    steps = 20
    g, (rho, ux, uy) = run(nx, ny, precision, variant, steps, RATES)
    oracle.set_mrt_rates(*RATES)
    try:
        ref = oracle.Lattice(nx, ny, 0.9)
        ref.init_density(rho, ux, uy)
        assert ref.step(steps, oracle.MRT, 0.8, 0.1)[0] == 0
    finally:
        oracle.set_mrt_rates(0.0, 0.0, 0.0)
    err = np.max(np.abs(g.populations() - ref.f)) / np.max(np.abs(ref.f))
    assert err < tol * steps ** 0.5, err


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64, lbm.BF16DEV])
def test_mrt_pair_kernel_matches_register_kernel_bitwise(precision):
    out = []
    for variant in (lbm.VARIANT_REGISTER, lbm.VARIANT_PAIR):
        g, _ = run(130, 41, precision, variant, 15, RATES)
        out.append((g.populations(), *g.observe()))
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_mrt_at_rates_one_over_tau_is_the_improved_scheme():
    """Default rates (1/tau): the same dynamics as LBM_SCHEME_IMPROVED up to
    FP32 rounding of the different operation order."""
    g, (rho, ux, uy) = run(64, 48, lbm.FP32, lbm.VARIANT_AUTO, 200, (0.0, 0.0, 0.0))
    h = lbm.Lattice(64, 48, 0.9, precision=lbm.FP32)
    h.init_density(rho, ux, uy)
    h.step(200, lbm.IMPROVED, 0.8, 0.1)
    assert np.max(np.abs(g.observe()[0] / h.observe()[0] - 1)) < 1e-5


def test_mrt_conserves_mass_and_rejects_bad_rates():
    g, _ = run(66, 40, lbm.FP64, lbm.VARIANT_AUTO, 0, RATES)
    m0 = g.mass()
    g.step(500, lbm.MRT, 0.8, 0.1)
    assert abs(g.mass() / m0 - 1) < 1e-13
    with pytest.raises(lbm.LbmError):
        g.set_mrt_rates(2.5, 1.0, 1.0)
    with pytest.raises(lbm.LbmError):
        g.set_mrt_rates(float("nan"), 1.0, 1.0)
