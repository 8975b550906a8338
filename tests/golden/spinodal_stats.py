"""Morphology-independent statistics of a phase-separating density field
(Sec. IV's spinodal decomposition workload), shared by the script that
writes the oracle's stored values and by the GPU test that compares against
them.  Pointwise values of a chaotic run differ between FP32 and FP64 after
a few hundred steps; the bulk densities of the two phases do not."""
import numpy as np


def bulk_densities(rho, rho_spinodal_lo, rho_spinodal_hi):
    """(vapour, liquid) bulk densities: medians of the cells below the lower
    and above the upper spinodal density (cells inside the spinodal are
    interface cells), and the fraction of cells in each set."""
    rho = np.asarray(rho)
    vap = rho[rho < rho_spinodal_lo]
    liq = rho[rho > rho_spinodal_hi]
    return {"rho_g": float(np.median(vap)) if vap.size else None,
            "rho_l": float(np.median(liq)) if liq.size else None,
            "frac_g": vap.size / rho.size, "frac_l": liq.size / rho.size}


def sample_grid(n, stride):
    """Cells (y, x) on a regular grid of the n x n lattice."""
    idx = np.arange(0, n, stride)
    return np.ix_(idx, idx)
