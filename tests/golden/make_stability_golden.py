"""Writes stability_oracle.json: the FP64 oracle's verdict (stable or not)
on the droplet of Figs. 1, 2 and 7 -- 200 x 200 periodic, Eq. 24 profile of
radius 30 and initial width W = 4 at the Maxwell densities of T (Tc = 0.094
as printed in Sec. III C), started at rest (zero actual velocity, Table I),
1e4 steps -- at the five reduced temperatures around each threshold the
paper prints: Shan-Chen, EDM and Guo's scheme (improved, sigma = 0) at
tau = 0.6 (Sec. IV B: unstable below 0.86, 0.73, 0.87), the improved scheme
with sigma = 0.105 at tau = 0.6 (stable from 0.63), EDM and EDM with
C_e = 1/tau at tau = 0.7 (Sec. III C: 0.67 and 0.57).  A run is unstable
when psi leaves its domain (divergence) or its largest actual speed exceeds
0.3 after the budget.  Calls only oracle/ and the input generator; run from
the repository root (a few minutes with the OpenMP build):

    python tests/golden/make_stability_golden.py
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

N, R0, W, STEPS, SPEED = 200, 30.0, 4.0, 10000, 0.3
# (name, scheme, sigma, tau, printed lowest stable T/Tc, where printed)
LADDERS = [
    ("SC", oracle.SC, 0.0, 0.6, 0.86, "Sec. IV B, after Fig. 7"),
    ("EDM", oracle.EDM, 0.0, 0.6, 0.73, "Sec. IV B, after Fig. 7"),
    ("GUO", oracle.IMPROVED, 0.0, 0.6, 0.87, "Sec. IV B, after Fig. 7"),
    ("IMPROVED_sigma0.105", oracle.IMPROVED, 0.105, 0.6, 0.63, "Sec. IV B, after Fig. 7"),
    ("EDM_tau0.7", oracle.EDM, 0.0, 0.7, 0.67, "Sec. III C, Fig. 2"),
    ("EDM_MOD_tau0.7", oracle.EDM_MOD, 0.0, 0.7, 0.57, "Sec. III C, Fig. 2"),
]


def verdict(lib, t, scheme, sigma, tau):
    eos = th.CarnahanStarling(th.temperature(t, 1))
    rg, rl, _ = th.maxwell(eos)
    lat = oracle.Lattice(N, N, t, tc_mode=1, lib=lib)
    lat.init_density_at_rest(inputs.droplet(N, N, rg, rl, R0, W=W))
    rc, done = lat.step(STEPS, scheme, tau, sigma)
    if rc:
        return False, done, None, rg, rl
    _, vx, vy = lat.observe()
    speed = float(np.sqrt(np.max(vx * vx + vy * vy)))
    return bool(speed <= SPEED), done, speed, rg, rl


def main():
    lib, threads = oracle.load_omp()
    out = {"_about": "FP64 oracle stability verdicts, droplet of Figs. 1, 2, 7: 200 x 200, "
                     "r0 = 30, W = 4, Maxwell densities with Tc = 0.094, at rest, 1e4 steps; "
                     "unstable = diverged or max |v| > 0.3; written by make_stability_golden.py",
           "n": N, "r0": R0, "W": W, "steps": STEPS, "speed_limit": SPEED, "tc_mode": 1,
           "ladders": []}
    for name, scheme, sigma, tau, printed, cite in LADDERS:
        pts = []
        for t in np.round(np.arange(printed + 0.02, printed - 0.0201, -0.01), 2):
            t0 = time.perf_counter()
            ok, done, speed, rg, rl = verdict(lib, float(t), scheme, sigma, tau)
            pts.append({"T_over_Tc": float(t), "stable": ok, "steps_done": done,
                        "max_speed": speed, "rho_g0": rg, "rho_l0": rl})
            print(name, t, ok, done, speed, f"{time.perf_counter() - t0:.0f} s ({threads} thr)",
                  flush=True)
        out["ladders"].append({"name": name, "scheme_id": scheme, "sigma": sigma, "tau": tau,
                               "printed_lowest_stable": printed, "cite": cite, "points": pts})
    with open(os.path.join(ROOT, "tests", "golden", "stability_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
