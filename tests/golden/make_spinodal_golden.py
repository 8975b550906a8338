"""Writes spinodal_1024_oracle.json: the FP64 oracle's spinodal decomposition
run at 1024 x 1024 (T = 0.85 Tc, tau = 0.8, improved scheme sigma = 0.1,
rho = rho_avg (1 + 0.01 U[-1, 1]) with seed 3, rho_avg the mean of the
Maxwell densities), the small-lattice version of the 8192^2 workload.

Stored: the density on a 32 x 32 grid of cells after 100 steps (pointwise
comparison while the run is still close to linear), the bulk densities of
both phases after 100 and 2000 steps, and the mass.  Calls only the oracle
and the seeded input generator.  Run time: several minutes (one core)."""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from oracle import theory as th  # noqa: E402
from paper_1204_4098_gb300 import inputs  # noqa: E402
from spinodal_stats import bulk_densities, sample_grid  # noqa: E402

N, T, TAU, SIGMA, SEED, STRIDE = 1024, 0.85, 0.8, 0.1, 3, 32


def main():
    eos = th.CarnahanStarling(th.temperature(T))
    rg, rl, _ = th.maxwell(eos)
    lo, hi = th.spinodal(eos)
    rho0 = inputs.spinodal(N, N, 0.5 * (rg + rl), amp=0.01, seed=SEED)
    lat = oracle.Lattice(N, N, T)
    lat.init_density(rho0)
    out = {"n": N, "T_over_Tc": T, "tau": TAU, "sigma": SIGMA, "seed": SEED, "stride": STRIDE,
           "spinodal": [lo, hi], "maxwell": [rg, rl], "mass0": float(lat.mass())}
    t0 = time.time()
    for target in (100, 2000):
        rc, _ = lat.step(target - lat.steps, oracle.IMPROVED, TAU, SIGMA)
        assert rc == 0, rc
        rho, _, _ = lat.observe()
        key = f"step{target}"
        out[key] = bulk_densities(rho, lo, hi)
        out[key]["mass"] = float(lat.mass())
        if target == 100:
            out[key]["rho_samples"] = rho[sample_grid(N, STRIDE)].tolist()
        print(target, out[key]["rho_g"], out[key]["rho_l"], f"{time.time() - t0:.0f} s",
              flush=True)
    with open(os.path.join(HERE, "spinodal_1024_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
