"""The C-ABI library without a GPU: it loads, exports every declared symbol,
rejects bad arguments before touching CUDA, and its host-side equation-of-
state helpers agree with the independent oracle theory tool."""
import ctypes
import os
import re
import subprocess

import pytest

from oracle import theory as th
from paper_1204_4098_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(lbm.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    return lbm.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_init_density", "lbm_step", "lbm_get_moments",
                     "lbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    names = declared_functions()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbm_[a-z0-9_]+)$", out, flags=re.M))
    assert set(names) <= exported, set(names) - exported


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) == set(lbm.SIGNATURES)


def test_params_struct_layout_matches(L):
    p = lbm.lbm_params()
    L.lbm_default_params(ctypes.byref(p))
    assert (p.a, p.b, p.R, p.G, p.precision, p.tc_mode) == (1.0, 4.0, 1.0, -1.0, 0, 0)
    assert p.cuda_stream is None


def test_create_rejects_bad_arguments_without_cuda(L):
    for kw in (dict(nx=0), dict(ny=-3), dict(T_over_Tc=0.0), dict(G=1.0), dict(precision=7),
               dict(tc_mode=5)):
        p = lbm.lbm_params()
        L.lbm_default_params(ctypes.byref(p))
        p.nx, p.ny, p.T_over_Tc = 8, 8, 0.8
        for k, v in kw.items():
            setattr(p, k, v)
        ctx = ctypes.c_void_p()
        st = L.lbm_create(ctypes.byref(p), ctypes.byref(ctx))
        assert st == lbm.LBM_E_INVAL, kw
        assert ctx.value is None
        assert L.lbm_last_error(None)


def test_null_context_calls_are_rejected(L):
    assert L.lbm_step(None, 1, 0, 1.0, 0.0) == lbm.LBM_E_INVAL
    assert L.lbm_set_mrt_rates(None, 1.0, 1.0, 1.0) == lbm.LBM_E_INVAL
    assert L.lbm_destroy(None) == lbm.LBM_OK


def test_wait_selftest_rejects_bad_arguments_without_cuda(L):
    r = ctypes.c_int(-1)
    assert L.lbm_selftest_wait_timeout(0, 0, ctypes.byref(r)) == lbm.LBM_E_INVAL
    assert L.lbm_selftest_wait_timeout(0, (1 << 20) + 1, ctypes.byref(r)) == lbm.LBM_E_INVAL
    assert L.lbm_selftest_wait_timeout(0, 10, None) == lbm.LBM_E_INVAL
    assert L.lbm_selftest_grid_barrier_timeout(0, None) == lbm.LBM_E_INVAL
    assert r.value == -1


def test_critical_point_matches_oracle(L):
    a = lbm.critical_point()
    b = th.critical_point()
    assert a == pytest.approx(b, rel=1e-13)


@pytest.mark.parametrize("t", [0.45, 0.55, 0.6, 0.7, 0.8, 0.85, 0.9, 0.95, 0.99])
def test_maxwell_matches_oracle(L, t):
    """Product: equal pressure and chemical potential (closed form, bisection);
    oracle: equal-area quadrature of Eq. 7."""
    got = lbm.maxwell(lbm.temperature(t))
    want = th.maxwell(th.CarnahanStarling(th.temperature(t)))
    assert got[0] == pytest.approx(want[0], rel=1e-10)
    assert got[1] == pytest.approx(want[1], rel=1e-12)


def test_maxwell_rejects_supercritical(L):
    with pytest.raises(lbm.LbmError):
        lbm.maxwell(lbm.critical_point()[1] * 1.01)


def test_batch_create_rejects_bad_arguments_without_cuda(L):
    good = dict(nx=8, ny=8, T_over_Tc=0.8, tau=1.0, sigma=0.0, scheme=0)
    for bad in (dict(nx=0), dict(ny=-1), dict(T_over_Tc=0.0), dict(tau=0.5), dict(scheme=9),
                dict(scheme=lbm.MRT), dict(sigma=float("nan"))):
        with pytest.raises(lbm.LbmError) as e:
            lbm.Batch([good, {**good, **bad}])
        assert e.value.status == lbm.LBM_E_INVAL
    for kw in (dict(window=3), dict(window=0), dict(max_steps=0), dict(mode=7), dict(conv=5),
               dict(conv_rel=-1e-6), dict(conv_rel=float("nan")), dict(variant=lbm.VARIANT_STAGED),
               dict(variant=9), dict(rows_per_item=-1)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.Batch([good], **kw)
        assert e.value.status == lbm.LBM_E_INVAL
    with pytest.raises(lbm.LbmError):
        lbm.Batch([])


def test_every_entry_point_is_documented():
    """Each declaration in include/lbm.h follows a comment (within three
    lines, so that a pair such as get/set populations can share one) that
    states what it does, its arguments and its errors."""
    lines = open(HEADER).read().splitlines()
    undocumented = []
    for i, line in enumerate(lines):
        m = re.match(r"\s*(?:lbm_status|const char \*|void|int)\s*\*?\s*(lbm_[a-z0-9_]+)\s*\(",
                     line)
        if m and not any("*/" in prev for prev in lines[max(0, i - 3):i]):
            undocumented.append(m.group(1))
    assert not undocumented, undocumented


def test_host_alloc_argument_checks_without_a_gpu(L):
    p = ctypes.c_void_p()
    assert L.lbm_host_alloc(0, ctypes.byref(p)) == lbm.LBM_E_INVAL
    assert L.lbm_host_alloc(64, None) == lbm.LBM_E_INVAL
    assert L.lbm_host_alloc(1 << 63, ctypes.byref(p)) == lbm.LBM_E_INVAL
    assert L.lbm_host_free(None) == lbm.LBM_OK
    scratch = ctypes.create_string_buffer(64)
    assert L.lbm_host_free(ctypes.cast(scratch, ctypes.c_void_p)) == lbm.LBM_E_INVAL
    # registration needs the CUDA driver: without a GPU the mapping is
    # returned and the status says so; with one, the buffer is usable
    st = L.lbm_host_alloc(4096, ctypes.byref(p))
    assert st in (lbm.LBM_OK, lbm.LBM_E_CUDA)
    if st == lbm.LBM_OK:
        assert L.lbm_host_free(p) == lbm.LBM_OK
    else:
        assert not p.value
