"""The y-slab decomposition on the GPU: band contexts (lbm_create_band) with
their halo rows packed, exchanged and unpacked after every step
(halo.LocalBands: several bands of one lattice on one GPU, exchanging by
device copies; one band is the periodic self-exchange).  Every owned row
evaluates what the same row of the undecomposed lattice evaluates, so the
results are compared bit for bit, with a droplet across the periodic wrap
in y (Eq. 1) and across band boundaries."""
import numpy as np
import pytest

from oracle import theory as th
from paper_1204_4098_gb300 import halo, inputs, lbm

pytestmark = pytest.mark.gpu

NX, T = 70, 0.85


def field(ny, seed=4):
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(T)))
    rho = inputs.droplet(NX, ny, rg, rl, 12.0, W=4.0, x0=NX / 2.0, y0=1.5)
    return rho


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("k", [1, 3, 4])
@pytest.mark.parametrize("precision,variant", [(lbm.FP32, lbm.VARIANT_PAIR),
                                               (lbm.FP32, lbm.VARIANT_REGISTER),
                                               (lbm.FP64, lbm.VARIANT_REGISTER),
                                               (lbm.BF16DEV, lbm.VARIANT_PAIR)])
def test_bands_match_whole_lattice_bitwise(k, precision, variant, overlap):
    ny, steps = 45, 40  # bands of 45, 15 and 11-12 rows
    rho = field(ny)
    whole = lbm.Lattice(NX, ny, T, precision=precision)
    whole.set_variant(variant)
    whole.init_density_at_rest(rho)
    whole.step(steps, lbm.IMPROVED, 0.8, 0.1)
    bands = halo.LocalBands(NX, ny, T, rho, k, precision=precision, at_rest=True)
    bands.set_variant(variant)
    assert bands.step(steps, lbm.IMPROVED, 0.8, 0.1, overlap=overlap) == lbm.LBM_OK
    assert np.array_equal(bands.populations(), whole.populations())
    for a, b in zip(bands.observe(), whole.observe()):
        assert np.array_equal(a, b)
    m = bands.mass()
    assert m == pytest.approx(whole.mass(), rel=1e-12)
    bands.close()


def test_band_contract():
    rho = field(20)
    b = lbm.Lattice(NX, 6, T, band=True)
    assert b.halo_bytes() == 2 * NX * 9 * 4
    with pytest.raises(AssertionError):
        b.init_density(rho[:6])  # a band's density carries two halo rows each side
    b.init_density(halo.with_halo(rho, 3, 6))
    with pytest.raises(lbm.LbmError) as e:
        b.step(2, lbm.SC, 1.0)  # one step per call: halos are exchanged between
    assert e.value.status == lbm.LBM_E_INVAL
    with pytest.raises(lbm.LbmError):
        b.set_populations(np.zeros((9, 6, NX)))
    assert b.populations().shape == (9, 6, NX) and b.observe()[0].shape == (6, NX)
    d = lbm.Lattice(NX, 6, T, precision=lbm.FP16DEV, band=True)
    assert d.halo_bytes() == 2 * NX * (9 * 2 + 4)
    whole = lbm.Lattice(NX, 6, T)
    with pytest.raises(lbm.LbmError) as e:
        whole.halo_bytes()
    assert e.value.status == lbm.LBM_E_STATE
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(NX, 1, T, band=True)  # a band owns at least two rows
    import torch
    buf = [torch.empty(b.halo_bytes(), dtype=torch.uint8, device="cuda") for _ in range(2)]
    lo, hi = buf[0].data_ptr(), buf[1].data_ptr()
    with pytest.raises(lbm.LbmError) as e:
        whole.step_overlap(lbm.SC, 1.0, 0.0, lo, hi)  # not a band
    assert e.value.status == lbm.LBM_E_STATE
    for bad in ((lbm.SC, 0.5, 0.0), (99, 1.0, 0.0), (lbm.SC, 1.0, float("nan"))):
        with pytest.raises(lbm.LbmError) as e:
            b.step_overlap(*bad, lo, hi)
        assert e.value.status == lbm.LBM_E_INVAL
    with pytest.raises(lbm.LbmError) as e:
        b.step_overlap(lbm.SC, 1.0, 0.0, 0, hi)  # no buffer
    assert e.value.status == lbm.LBM_E_INVAL
    fresh = lbm.Lattice(NX, 6, T, band=True)
    with pytest.raises(lbm.LbmError) as e:
        fresh.step_overlap(lbm.SC, 1.0, 0.0, lo, hi)  # not initialised
    assert e.value.status == lbm.LBM_E_STATE


def test_band_runner_with_overlap_matches_whole_lattice():
    """halo.BandLattice (the multi-rank runner) on one rank: the boundary
    rows first, the exchange on its own stream (here the periodic
    self-exchange) while the interior rows run, the unpack before the next
    step -- bit-identical to the whole lattice, for a band thin enough to
    have no interior as well."""
    for ny in (45, 4):
        rho = field(ny)
        whole = lbm.Lattice(NX, ny, T, precision=lbm.FP32)
        whole.set_variant(lbm.VARIANT_PAIR)
        whole.init_density(rho)
        whole.step(30, lbm.EDM, 0.7)
        band = halo.BandLattice(NX, ny, T, rho)
        band.lat.set_variant(lbm.VARIANT_PAIR)
        assert band.step(30, lbm.EDM, 0.7, overlap=True) == lbm.LBM_OK
        for a, b in zip(band.observe(), whole.observe()):
            assert np.array_equal(a, b), ny
        band.close()


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.BF16DEV])
def test_bands_with_odd_width_match_whole_lattice_bitwise(precision):
    """Odd nx runs on the one-column kernel; its bands carry the same two
    ghost rows and exchange the same messages (width nx)."""
    nx, ny, steps = 71, 38, 25
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(T)))
    rho = inputs.droplet(nx, ny, rg, rl, 11.0, W=4.0, x0=nx / 2.0, y0=ny - 2.0)
    whole = lbm.Lattice(nx, ny, T, precision=precision)
    whole.init_density_at_rest(rho)
    whole.step(steps, lbm.EDM, 0.7)
    for overlap in (False, True):
        bands = halo.LocalBands(nx, ny, T, rho, 3, precision=precision, at_rest=True)
        assert bands.step(steps, lbm.EDM, 0.7, overlap=overlap) == lbm.LBM_OK
        assert np.array_equal(bands.populations(), whole.populations())
        bands.close()
