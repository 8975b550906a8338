"""Spinodal decomposition at 1024 x 1024 (the 8192^2 workload's recipe on a
lattice the FP64 oracle finishes in minutes) against the oracle's stored run
(tests/golden/spinodal_1024_oracle.json, written by make_spinodal_golden.py).

The run is chaotic: FP32 and FP64 separate pointwise after a few hundred
steps, so the pointwise comparison is made at step 100, and after 2000 steps
the bulk densities of the two phases (medians outside the spinodal) are
compared, which coarsening does not make chaotic."""
import json
import os
import sys

import numpy as np
import pytest

from paper_1204_4098_gb300 import inputs, lbm

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from spinodal_stats import bulk_densities, sample_grid  # noqa: E402

pytestmark = pytest.mark.gpu

with open(os.path.join(os.path.dirname(__file__), "golden", "spinodal_1024_oracle.json")) as _f:
    GOLD = json.load(_f)


def start(precision):
    n = GOLD["n"]
    rg, rl = GOLD["maxwell"]
    rho0 = inputs.spinodal(n, n, 0.5 * (rg + rl), amp=0.01, seed=GOLD["seed"])
    lat = lbm.Lattice(n, n, GOLD["T_over_Tc"], precision=precision)
    lat.init_density(rho0)
    return lat


def advance(lat, steps):
    lat.step(steps, lbm.IMPROVED, GOLD["tau"], GOLD["sigma"])
    return lat.observe()[0]


def test_spinodal_1024_fp32_against_oracle():
    lat = start(lbm.FP32)
    m0 = lat.mass()
    assert m0 == pytest.approx(GOLD["mass0"], rel=1e-7)
    rho = advance(lat, 100)
    want = np.array(GOLD["step100"]["rho_samples"])
    got = rho[sample_grid(GOLD["n"], GOLD["stride"])]
    err = np.max(np.abs(got / want - 1))
    print(f"step 100: max rel err {err:.2e} over {want.size} cells")
    assert err <= 1e-4
    rho = advance(lat, 1900)
    lo, hi = GOLD["spinodal"]
    got = bulk_densities(rho, lo, hi)
    ref = GOLD["step2000"]
    print("step 2000 bulk densities: gpu", got, "oracle", ref)
    assert got["rho_l"] == pytest.approx(ref["rho_l"], rel=1e-3)
    assert got["rho_g"] == pytest.approx(ref["rho_g"], rel=1e-3)
    assert abs(lat.mass() / m0 - 1) < 1e-6


@pytest.mark.parametrize("precision,tol", [(lbm.FP16DEV, 2e-3), (lbm.BF16DEV, 1e-2)])
def test_spinodal_1024_16bit_bulk_densities(precision, tol):
    """16-bit deviation storage: the bulk densities after 2000 steps, against
    the FP64 oracle.  The gate is the deviation's rounding carried to the
    density (fp16: 11-bit, bf16: 8-bit significand of deviations of a few
    per cent of rho, i.e. ~1e-5 and ~1e-4 per step on a population) with the
    margin the FP32 run needs for coarsening (1e-3)."""
    lat = start(precision)
    rho = advance(lat, 2000)
    lo, hi = GOLD["spinodal"]
    got = bulk_densities(rho, lo, hi)
    ref = GOLD["step2000"]
    err = max(abs(got["rho_l"] / ref["rho_l"] - 1), abs(got["rho_g"] / ref["rho_g"] - 1))
    print(f"16-bit storage {precision}: bulk densities {got}, max rel err vs oracle {err:.2e}")
    assert err < tol
