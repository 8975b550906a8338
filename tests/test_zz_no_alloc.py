"""The allocation-free mass entry point against lbm_get_mass and an FP64 sum.

lbm_mass_f32_noalloc serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or they must not block on an
allocation): it sums an FP32 buffer the caller owns into a device slot the
caller owns, using a fixed file-scope scratch array.  This file is collected
last, so a stop-at-first-failure run has executed every other test before it.
"""
import ctypes

import numpy as np
import pytest

from oracle import theory as th
from paper_1204_4098_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


def _noalloc_sum(torch, f, out):
    st = lbm.lib().lbm_mass_f32_noalloc(ctypes.c_void_p(f.data_ptr()), f.numel(),
                                         ctypes.c_void_p(out.data_ptr()), None)
    assert st == lbm.LBM_OK
    torch.cuda.synchronize()
    return float(out.item())


def test_mass_noalloc_matches_lbm_get_mass_on_two_calls():
    torch = pytest.importorskip("torch")
    nx, ny, t = 70, 50, 0.85
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(t)))
    lat = lbm.Lattice(nx, ny, t, precision=lbm.FP32)
    lat.init_density(inputs.droplet(nx, ny, rg, rl, 12.0, W=4.0))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        lat.step(50 + 25 * call, lbm.IMPROVED, 0.8, 0.1)
        want = lat.mass()  # existing entry point (context-owned scratch)
        f = torch.tensor(lat.populations(), dtype=torch.float32, device="cuda").contiguous()
        torch.cuda.synchronize()
        got = _noalloc_sum(torch, f, out)
        # both are FP64 sums of the same FP32 values, in different orders
        assert got == pytest.approx(want, rel=1e-12), (call, got, want)


@pytest.mark.parametrize("n", [1, 4095, 4096, 4097, 1 << 20, (1 << 20) + 1,
                               3 * (1 << 20) + 17])
def test_mass_noalloc_multi_block_against_fp64_sum(n):
    """Sizes on both sides of the per-block minimum (4096 values) and well
    past it (up to 768 blocks), on two calls in a row with different data,
    against numpy's FP64 sum of the same FP32 values."""
    torch = pytest.importorskip("torch")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(n)
    for call in range(2):
        x = rng.uniform(0.0, 1.0, n).astype(np.float32)
        f = torch.from_numpy(x).to("cuda")
        want = float(np.sum(x.astype(np.float64)))
        got = _noalloc_sum(torch, f, out)
        assert got == pytest.approx(want, rel=1e-12), (n, call, got, want)


def test_mass_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = lbm.lib()
    assert L.lbm_mass_f32_noalloc(None, 10, ctypes.c_void_p(out.data_ptr()), None) == \
        lbm.LBM_E_INVAL
    assert L.lbm_mass_f32_noalloc(ctypes.c_void_p(out.data_ptr()), (1 << 30) + 1,
                                  ctypes.c_void_p(out.data_ptr()), None) == lbm.LBM_E_INVAL
    assert L.lbm_mass_f32_noalloc(None, 0, ctypes.c_void_p(out.data_ptr()), None) == lbm.LBM_OK
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
