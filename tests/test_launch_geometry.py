"""The single-lattice launch rules without a GPU
(paper_1204_4098_gb300/csrc/lbm_geometry.h, compiled with the host C++
compiler through tests/host_shim.cpp): which kernel variant a context
resolves to, and the warp-strip geometry of one wave."""
import ctypes

import numpy as np
import pytest

from paper_1204_4098_gb300 import lbm

AUTO, REG, STAGED, PAIR = (lbm.VARIANT_AUTO, lbm.VARIANT_REGISTER, lbm.VARIANT_STAGED,
                           lbm.VARIANT_PAIR)
SMS = 152  # GB300


def variant(S, requested, precision, nx, ny, step=True):
    return S.shim_resolve_variant(requested, precision, nx, ny, SMS, 1 if step else 0)


def geometry(S, nx, ny, var, resident, wpc=4, override=0):
    out = (ctypes.c_int * 4)()
    S.shim_strip_geometry(nx, ny, var, resident, wpc, override, out)
    return dict(n_strips=out[0], band_rows=out[1], n_bands=out[2], grid=out[3])


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.BF16DEV, lbm.FP16DEV])
def test_auto_takes_two_columns_for_even_nx(host_shim, precision):
    assert variant(host_shim, AUTO, precision, 8192, 8192) == PAIR
    assert variant(host_shim, AUTO, precision, 8191, 8192) == REG  # odd nx
    assert variant(host_shim, AUTO, precision, 8192, 8192, step=False) == PAIR  # observe too


def test_auto_keeps_one_column_in_fp64(host_shim):
    assert variant(host_shim, AUTO, lbm.FP64, 8192, 8192) == REG
    # an explicit request is honoured (it spills, but it runs)
    assert variant(host_shim, PAIR, lbm.FP64, 8192, 8192) == PAIR


def test_auto_keeps_one_column_on_small_lattices(host_shim):
    # 256^2 measured faster with one column per lane, 512^2 and up with two:
    # the rule compares the two-column items (64-column strips x 4-row bands)
    # with a quarter of the resident warps (152 SMs x 20)
    assert variant(host_shim, AUTO, lbm.FP32, 256, 256) == REG
    assert variant(host_shim, AUTO, lbm.FP32, 512, 512) == PAIR
    items = lambda n: ((n + 63) // 64) * ((n + 3) // 4)  # noqa: E731
    for n in range(64, 1025, 8):
        want = REG if items(n) * 4 < SMS * 20 else PAIR
        assert variant(host_shim, AUTO, lbm.FP32, n, n) == want, n


def test_staged_only_where_its_copies_are_aligned(host_shim):
    assert variant(host_shim, STAGED, lbm.FP32, 4096, 4096) == STAGED
    assert variant(host_shim, STAGED, lbm.FP32, 4098, 64) == REG  # nx % 4 != 0
    assert variant(host_shim, STAGED, lbm.FP32, 60, 64) == REG  # nx < 64
    assert variant(host_shim, STAGED, lbm.FP64, 4096, 4096) == REG
    assert variant(host_shim, STAGED, lbm.BF16DEV, 4096, 4096) == REG
    assert variant(host_shim, STAGED, lbm.FP32, 4096, 4096, step=False) == REG  # observe


def test_requested_variants(host_shim):
    assert variant(host_shim, REG, lbm.FP32, 8192, 8192) == REG
    assert variant(host_shim, PAIR, lbm.FP32, 256, 256) == PAIR  # small, but asked for
    assert variant(host_shim, PAIR, lbm.FP32, 255, 256) == REG  # odd nx cannot pair


def test_bench_geometry_is_one_wave(host_shim):
    # 8192^2 with the two-column kernel at 4 CTAs of 4 warps per SM
    g = geometry(host_shim, 8192, 8192, PAIR, SMS * 4 * 4)
    assert g == dict(n_strips=128, band_rows=432, n_bands=19, grid=608)


@pytest.mark.parametrize("seed", range(5))
def test_geometry_covers_the_lattice_in_one_wave(host_shim, seed):
    rng = np.random.default_rng(seed)
    for _ in range(200):
        nx, ny = (int(v) for v in rng.integers(1, 5000, 2))
        var = PAIR if rng.random() < 0.5 else REG
        resident = int(rng.integers(1, 8)) * SMS * 4
        g = geometry(host_shim, nx, ny, var, resident)
        w = 64 if var == PAIR else 32
        assert g["n_strips"] == (nx + w - 1) // w
        # the bands tile the rows exactly once
        assert g["n_bands"] * g["band_rows"] >= ny > (g["n_bands"] - 1) * g["band_rows"]
        assert g["band_rows"] >= min(host_shim.shim_min_band_rows(nx, ny), ny)
        # one wave, unless the strips alone exceed it
        items = g["n_strips"] * g["n_bands"]
        assert items <= max(resident, g["n_strips"])
        # one warp per item
        assert (g["grid"] - 1) * 4 < items <= g["grid"] * 4


def test_small_lattices_take_the_shortest_bands(host_shim):
    # the step of a small lattice is one short wave: 1-row bands up to 128^2
    # cells, 2-row bands up to 256^2, then at least 4 rows
    assert [host_shim.shim_min_band_rows(n, n) for n in (64, 128, 129, 256, 257, 512)] == \
        [1, 1, 2, 2, 4, 4]
    for n, rows in ((64, 1), (128, 1), (256, 2), (512, 4)):
        g = geometry(host_shim, n, n, REG, SMS * 6 * 4)
        assert g["band_rows"] == rows and g["n_bands"] == n // rows, n
    g = geometry(host_shim, 4096, 4096, PAIR, SMS * 4 * 4)  # one wave, taller bands
    assert g["band_rows"] > 4


def test_band_height_override(host_shim):
    g = geometry(host_shim, 1000, 300, REG, SMS * 24, override=64)
    assert g["band_rows"] == 64 and g["n_bands"] == 5
    g = geometry(host_shim, 1000, 30, REG, SMS * 24, override=64)
    assert g["band_rows"] == 30 and g["n_bands"] == 1
    assert geometry(host_shim, 1, 1, REG, SMS * 24) == dict(n_strips=1, band_rows=1, n_bands=1,
                                                           grid=1)
