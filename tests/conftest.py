import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU oracle physics run")


@pytest.fixture(scope="session")
def host_shim(tmp_path_factory):
    """tests/host_shim.cpp (the library's host-side rules, plain C++) built
    with the host compiler and loaded through ctypes."""
    import ctypes
    import shutil
    import subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("shim") / "libhostshim.so")
    subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1204_4098_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_shim.cpp"), "-o", out],
                   check=True, capture_output=True, text=True)
    lib = ctypes.CDLL(out)
    P, I = ctypes.c_void_p, ctypes.c_int
    IP = ctypes.POINTER(ctypes.c_int)
    lib.shim_tuner_new.restype = P
    lib.shim_tuner_free.argtypes = [P]
    lib.shim_tuner_add.argtypes = [P, I, I]
    lib.shim_tuner_choose.argtypes = [P, ctypes.c_ulonglong, IP, IP, IP]
    lib.shim_tuner_record.argtypes = [P, I, I, ctypes.c_double]
    lib.shim_tuner_disable.argtypes = [P, I]
    lib.shim_tuner_tuned.argtypes = [P]
    lib.shim_lpt.argtypes = [I, ctypes.POINTER(ctypes.c_longlong), I, IP, IP]
    lib.shim_resolve_variant.argtypes = [I, I, I, I, I, I]
    D = ctypes.c_double
    lib.shim_window_verdict.argtypes = [I, D, D, I, I, ctypes.POINTER(D), I, I, I, IP,
                                        ctypes.c_void_p]
    lib.shim_window_verdict_trend.argtypes = [D, D, I, I, ctypes.POINTER(D), I,
                                              ctypes.POINTER(D), ctypes.c_void_p]
    lib.shim_trend_remaining.argtypes = [D, D]
    lib.shim_trend_remaining.restype = D
    lib.shim_trend_hist.restype = I
    lib.shim_strip_geometry.argtypes = [I, I, I, ctypes.c_longlong, I, I, IP]
    return lib
