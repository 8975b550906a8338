"""Calibration of sigma against the Maxwell construction (Sec. IV B) on the
batch engine, against the FP64 oracle's mechanical-stability theory (Eq. 26
with eps = 16 sigma) and the paper's fitted sigma = 0.105."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import theory as th
from paper_1204_4098_gb300 import calibrate

pytestmark = pytest.mark.gpu

PAPER_SIGMA = 0.105  # Sec. IV B: sigma = 0.105 (eps = 1.68) fits the Maxwell construction


def theory_sigma_star(t):
    """sigma where the mechanical-stability vapour density equals Maxwell's."""
    eos = th.CarnahanStarling(th.temperature(t))
    rg = th.maxwell(eos)[0]
    return brentq(lambda s: th.mechanical_stability(eos, 16.0 * s)[0] - rg, 0.07, 0.2,
                  xtol=1e-10)


def test_sigma_calibration():
    """sigma*(T) from converged slabs agrees with the theory within 0.01 (the
    theory is truncated at second order; 0.01 in sigma is the 5 % in rho_g
    the flat-interface pin allows) and brackets the paper's 0.105."""
    temps = (0.7, 0.8, 0.9)
    out, info = calibrate.sigma_star(temps, sigmas=np.arange(0.08, 0.1351, 0.01), refine=3)
    stars = []
    for row in out:
        s_th = theory_sigma_star(row["T_over_Tc"])
        print(row["T_over_Tc"], "sigma* simulated", row["sigma_star"], "theory", s_th)
        assert row["sigma_star"] is not None
        assert abs(row["sigma_star"] - s_th) < 0.01
        stars.append(row["sigma_star"])
    print("gpu s", info["gpu_s"])
    assert abs(np.mean(stars) - PAPER_SIGMA) < 0.01
