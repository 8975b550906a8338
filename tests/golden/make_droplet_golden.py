"""Writes droplets_256_oracle.json: config 2's static droplet (256 x 256
periodic, Eq. 24 profile of radius 30 and width 5 at the Maxwell densities,
at rest u = 0, T = 0.8 Tc, exact Tc) run 2e4 steps by the FP64 oracle for
one point per forcing scheme: Shan-Chen (Eqs. 9-10) and the improved scheme
(Eq. 31, sigma = 0.1) at tau = 1, EDM (Eq. 11) and the improved scheme at
the paper's sigma = 0.105 at tau = 0.6.  Stored: the initial densities and
the droplet observables (centre and corner densities, equivalent-area
radius, pressure jump of Eq. 23, largest actual speed).  Calls only oracle/
and the seed-free input generator; run from the repository root:

    python tests/golden/make_droplet_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import theory as th  # noqa: E402
from paper_1204_4098_gb300 import inputs  # noqa: E402

N, R0, W, T_OVER_TC, STEPS = 256, 30.0, 5.0, 0.8, 20000
POINTS = [("SC", oracle.SC, 1.0, 0.0), ("EDM", oracle.EDM, 0.6, 0.0),
          ("IMPROVED", oracle.IMPROVED, 1.0, 0.1), ("IMPROVED", oracle.IMPROVED, 0.6, 0.105)]


def observables(rho, vx, vy, T):
    """Centre / corner densities, equivalent-area radius, Eq. 23 pressure jump."""
    ny, nx = rho.shape
    r_in, r_out = float(rho[ny // 2, nx // 2]), float(rho[0, 0])
    cs = th.CarnahanStarling(T)
    return {"rho_in": r_in, "rho_out": r_out,
            "radius": float(np.sqrt(np.sum(rho - r_out) / (r_in - r_out) / np.pi)),
            "dp": float(cs.p(r_in) - cs.p(r_out)),
            "max_speed": float(np.sqrt(np.max(vx * vx + vy * vy)))}


def main():
    T = th.temperature(T_OVER_TC)
    rg, rl, _ = th.maxwell(th.CarnahanStarling(T))
    lib, threads = oracle.load_omp()
    out = {"_about": "FP64 oracle, config 2 droplet: 256 x 256 periodic, Eq. 24 (r0 = 30, "
                     "W = 5, centre (nx/2, ny/2)) at the Maxwell densities, u = 0, "
                     "T = 0.8 Tc (exact Tc), 2e4 steps; written by make_droplet_golden.py",
           "n": N, "r0": R0, "W": W, "T_over_Tc": T_OVER_TC, "steps": STEPS,
           "rho_g0": rg, "rho_l0": rl, "points": []}
    rho0 = inputs.droplet(N, N, rg, rl, R0, W=W)
    for name, scheme, tau, sigma in POINTS:
        t0 = time.perf_counter()
        lat = oracle.Lattice(N, N, T_OVER_TC, lib=lib)
        lat.init_density(rho0)
        rc, done = lat.step(STEPS, scheme, tau, sigma)
        assert rc == 0 and done == STEPS, (name, rc, done)
        obs = observables(*lat.observe(), T)
        out["points"].append({"scheme": name, "scheme_id": scheme, "tau": tau, "sigma": sigma,
                              **obs})
        print(name, tau, sigma, obs, f"{time.perf_counter() - t0:.0f} s ({threads} threads)",
              flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "droplets_256_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
