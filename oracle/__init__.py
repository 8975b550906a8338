"""FP64 CPU oracle of the pseudopotential D2Q9 lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_1204_4098_gb300`` and neither imports
the other; the two meet only in the seeded input generators of
``paper_1204_4098_gb300.inputs``, which hold none of the method's arithmetic.

* ``lbm_oracle.c`` -- the time step, written out step by step in FP64 plain C
  (moments, Eq. 8/23 potential, Eq. 3 force, the forcing schemes of Eqs. 9-11,
  12-13, 31 and Table I, streaming of Eq. 1).  Loaded here through ctypes.
* ``theory.py`` -- critical point, Maxwell construction (Eq. 7) and the
  mechanical-stability condition (Eqs. 6, 26, 30).

Parity status of each function is recorded in its test module; every
function here is pinned by a CPU test against something other than itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import theory

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
# the same source built with -fopenmp (cell loops split over threads,
# bit-identical results); used to time the oracle on all host cores
_LIB_OMP = os.path.join(_HERE, "liblbm_oracle_omp.so")

SC, EDM, IMPROVED, NOFORCE, EDM_MOD, LADD, MRT = range(7)
Q = 9
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def compile_oracle(src: str = _SRC, out: str = _LIB, defines=(), openmp=False) -> str:
    """Compile the C oracle with gcc (FP contraction off, so x86 and Arm hosts
    round identically); ``openmp`` adds -fopenmp."""
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           *(["-fopenmp"] if openmp else []),
           *[f"-D{d}" for d in defines], "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def compile_all() -> None:
    """Both builds: plain (single-threaded) and OpenMP (if gcc supports it)."""
    compile_oracle()
    try:
        compile_oracle(out=_LIB_OMP, openmp=True)
    except (subprocess.CalledProcessError, OSError):
        pass


def _declare(lib):
    d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    sig = {
        "oracle_version": (i, []),
        "oracle_threads": (i, [i]),
        "oracle_p_eos": (d, [d, d, d, d]),
        "oracle_psi": (i, [d, d, d, d, d, p]),
        "oracle_feq": (None, [d, d, d, p]),
        "oracle_moments": (None, [i, i, p, p, p, p]),
        "oracle_psi_field": (i, [i, i, p, d, d, d, d, p]),
        "oracle_force": (None, [i, i, d, p, p, p]),
        "oracle_collide_cell": (i, [i, d, d, p, d, d, d, p]),
        "oracle_set_mrt_rates": (None, [d, d, d]),
        "oracle_stream": (None, [i, i, p, p]),
        "oracle_step": (i, [i, i, p, i, d, d, d, d, d, d]),
        "oracle_run": (i, [i, i, p, i, i, d, d, d, d, d, d, p]),
        "oracle_init_equilibrium": (None, [i, i, p, p, p, p]),
        "oracle_init_at_rest": (i, [i, i, p, d, d, d, d, p]),
        "oracle_observe": (i, [i, i, p, d, d, d, d, i, p, p, p]),
        "oracle_mass": (d, [i, i, p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib_cache = {}


def load(path: str = _LIB):
    """The oracle library (compiled on first use if it is missing)."""
    if path not in _lib_cache:
        if path in (_LIB, _LIB_OMP) and (not os.path.exists(path)
                                         or os.path.getmtime(path) < os.path.getmtime(_SRC)):
            compile_oracle(out=path, openmp=path == _LIB_OMP)
        _lib_cache[path] = _declare(ctypes.CDLL(path))
    return _lib_cache[path]


def load_omp(threads: int = 0):
    """The OpenMP build (None if it cannot be built); ``threads`` > 0 sets
    its thread count.  Returns (library, threads in use)."""
    try:
        lib = load(_LIB_OMP)
    except (subprocess.CalledProcessError, OSError):
        return None, 1
    return lib, lib.oracle_threads(int(threads))


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _vec(x):
    return np.ascontiguousarray(x, dtype=np.float64)


# ---------------------------------------------------------------------------
# pointwise helpers
# ---------------------------------------------------------------------------

def p_eos(rho, RT, a=1.0, b=4.0, lib=None):
    lib = lib or load()
    return lib.oracle_p_eos(float(rho), RT, a, b)


def psi(rho, RT, a=1.0, b=4.0, G=-1.0, lib=None):
    lib = lib or load()
    out = ctypes.c_double()
    rc = lib.oracle_psi(float(rho), RT, a, b, G, ctypes.byref(out))
    return None if rc else out.value


def feq(rho, ux, uy, lib=None):
    lib = lib or load()
    out = np.zeros(Q)
    lib.oracle_feq(float(rho), float(ux), float(uy), _ptr(out))
    return out


def set_mrt_rates(s_e=0.0, s_eps=0.0, s_q=0.0, lib=None):
    """Relaxation rates of the MRT scheme's energy, energy-square and
    energy-flux moments (<= 0: 1/tau); process-wide."""
    lib = lib or load()
    lib.oracle_set_mrt_rates(float(s_e), float(s_eps), float(s_q))


def collide_cell(scheme, tau, sigma, f, Fx, Fy, psi_c=1.0, lib=None):
    lib = lib or load()
    f = _vec(f)
    out = np.zeros(Q)
    rc = lib.oracle_collide_cell(int(scheme), float(tau), float(sigma), _ptr(f),
                                 float(Fx), float(Fy), float(psi_c), _ptr(out))
    if rc:
        raise ValueError("unknown scheme")
    return out


def force(psi_field, G=-1.0, lib=None):
    lib = lib or load()
    psi_field = _vec(psi_field)
    ny, nx = psi_field.shape
    Fx, Fy = np.zeros_like(psi_field), np.zeros_like(psi_field)
    lib.oracle_force(nx, ny, G, _ptr(psi_field), _ptr(Fx), _ptr(Fy))
    return Fx, Fy


def stream(fpost, lib=None):
    lib = lib or load()
    fpost = _vec(fpost)
    _, ny, nx = fpost.shape
    out = np.zeros_like(fpost)
    lib.oracle_stream(nx, ny, _ptr(fpost), _ptr(out))
    return out


def moments(f, lib=None):
    lib = lib or load()
    f = _vec(f)
    _, ny, nx = f.shape
    rho, ux, uy = (np.zeros((ny, nx)) for _ in range(3))
    lib.oracle_moments(nx, ny, _ptr(f), _ptr(rho), _ptr(ux), _ptr(uy))
    return rho, ux, uy


def init_equilibrium(rho, ux=None, uy=None, lib=None):
    lib = lib or load()
    rho = _vec(rho)
    ny, nx = rho.shape
    f = np.zeros((Q, ny, nx))
    ux = None if ux is None else _vec(ux)
    uy = None if uy is None else _vec(uy)
    lib.oracle_init_equilibrium(nx, ny, _ptr(rho),
                                None if ux is None else _ptr(ux),
                                None if uy is None else _ptr(uy), _ptr(f))
    return f


# ---------------------------------------------------------------------------
# a lattice with the same life cycle as the C-ABI (create, init, step, observe)
# ---------------------------------------------------------------------------

class Lattice:
    """FP64 oracle state with the same life cycle as the CUDA C-ABI."""

    def __init__(self, nx, ny, T_over_Tc, tc_mode=0, a=1.0, b=4.0, R=1.0,
                 G=-1.0, lib=None):
        self.nx, self.ny = int(nx), int(ny)
        self.a, self.b, self.R, self.G = a, b, R, G
        self.T = theory.temperature(T_over_Tc, tc_mode, a, b, R)
        self.RT = R * self.T
        self.lib = lib or load()
        self.f = np.zeros((Q, self.ny, self.nx))
        self.steps = 0
        self.last_scheme = SC

    def init_density(self, rho, ux=None, uy=None):
        self.f = init_equilibrium(rho, ux, uy, lib=self.lib)
        self.steps = 0

    def init_density_at_rest(self, rho):
        """f = f_eq(rho, u) with u = -F / (2 rho) (zero actual velocity)."""
        rho = _vec(rho)
        assert rho.shape == (self.ny, self.nx)
        f = np.zeros((Q, self.ny, self.nx))
        rc = self.lib.oracle_init_at_rest(self.nx, self.ny, _ptr(rho), self.RT, self.a,
                                          self.b, self.G, _ptr(f))
        if rc:
            raise FloatingPointError("density outside the domain of psi")
        self.f = f
        self.steps = 0

    def step(self, n, scheme, tau, sigma=0.0):
        """Advance n steps; returns (status, completed_steps)."""
        done = ctypes.c_int(0)
        rc = self.lib.oracle_run(self.nx, self.ny, _ptr(self.f), int(n),
                                 int(scheme), float(tau), float(sigma), self.RT,
                                 self.a, self.b, self.G, ctypes.byref(done))
        self.steps += done.value
        self.last_scheme = scheme
        return rc, done.value

    def observe(self, noforce=None):
        """(rho, vx, vy) with v = u + F/(2 rho) from the current state."""
        if noforce is None:
            noforce = self.last_scheme == NOFORCE
        rho, vx, vy = (np.zeros((self.ny, self.nx)) for _ in range(3))
        rc = self.lib.oracle_observe(self.nx, self.ny, _ptr(self.f), self.RT,
                                     self.a, self.b, self.G, int(bool(noforce)),
                                     _ptr(rho), _ptr(vx), _ptr(vy))
        if rc:
            raise FloatingPointError("density outside the domain of psi")
        return rho, vx, vy

    def mass(self):
        return self.lib.oracle_mass(self.nx, self.ny, _ptr(self.f))
