"""The oracle's OpenMP build (cell loops split over threads) against its
plain single-threaded build: bit-identical populations for every scheme,
and the same divergence status.  The OpenMP build exists to time the oracle
on all host cores; it must not change a single bit of what it computes."""
import numpy as np
import pytest

import oracle
from oracle import theory as th
from paper_1204_4098_gb300 import inputs


def _omp(threads):
    lib, n = oracle.load_omp(threads)
    if lib is None:
        pytest.skip("gcc has no OpenMP here")
    return lib, n


@pytest.mark.parametrize("scheme,sigma", [(oracle.SC, 0.0), (oracle.EDM, 0.0),
                                          (oracle.IMPROVED, 0.1), (oracle.NOFORCE, 0.0),
                                          (oracle.EDM_MOD, 0.0), (oracle.LADD, 0.0),
                                          (oracle.MRT, 0.1)])
def test_openmp_build_bit_identical(scheme, sigma):
    nx, ny, t = 67, 45, 0.85  # odd sizes: rows and cells do not split evenly
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(t)))
    rho0 = inputs.spinodal(nx, ny, 0.5 * (rg + rl), amp=0.01, seed=3)
    libo, n = _omp(3)
    out = []
    for lib in (oracle.load(), libo):
        lat = oracle.Lattice(nx, ny, t, lib=lib)
        lat.init_density(rho0)
        rc, done = lat.step(15, scheme, 0.8, sigma)
        assert (rc, done) == (0, 15)
        out.append((lat.f.copy(), lat.observe()))
    assert np.array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)


def test_openmp_build_reports_divergence_like_the_plain_build():
    nx, ny, t = 40, 30, 0.85
    rho = np.full((ny, nx), 0.2)
    rho[7, 11] = 1.5  # b rho / 4 >= 1: outside the domain of psi
    libo, _ = _omp(4)
    res = []
    for lib in (oracle.load(), libo):
        lat = oracle.Lattice(nx, ny, t, lib=lib)
        lat.init_density(rho)
        f0 = lat.f.copy()
        res.append(lat.step(3, oracle.IMPROVED, 0.8, 0.1))
        assert np.array_equal(lat.f, f0)  # a diverged step leaves f unchanged
    assert res[0] == res[1] == (1, 0)


def test_openmp_thread_count_is_settable():
    _, n = _omp(2)
    assert n == 2
    assert oracle.load().oracle_threads(5) == 1  # the plain build has one thread
