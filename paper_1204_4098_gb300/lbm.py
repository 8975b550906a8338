"""Thin ctypes binding of the C ABI declared in ``include/lbm.h``.

Argument marshalling only: every function forwards to the function of the
same name in ``liblbm_gb300.so``, and every step of the method runs in that
library's CUDA kernels.  There is no fallback: if the library is missing the
first call raises, telling how to build it.

``Lattice`` is a small convenience wrapper (numpy arrays in and out, errors
raised as ``LbmError``) over the same calls.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_gb300.so")

LBM_OK, LBM_E_INVAL, LBM_E_NOMEM, LBM_E_CUDA, LBM_E_DIVERGED, LBM_E_TIMEOUT, LBM_E_STATE = range(7)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_E_INVAL", 2: "LBM_E_NOMEM", 3: "LBM_E_CUDA",
                4: "LBM_E_DIVERGED", 5: "LBM_E_TIMEOUT", 6: "LBM_E_STATE"}
SC, EDM, IMPROVED, NOFORCE, EDM_MOD, LADD, MRT = range(7)
FP32, FP64, BF16DEV, FP16DEV = range(4)
VARIANT_AUTO, VARIANT_REGISTER, VARIANT_STAGED, VARIANT_PAIR = range(4)


class lbm_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("T_over_Tc", ctypes.c_double), ("tc_mode", ctypes.c_int),
                ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("R", ctypes.c_double), ("G", ctypes.c_double),
                ("precision", ctypes.c_int), ("device", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


class lbm_instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("T_over_Tc", ctypes.c_double),
                ("tau", ctypes.c_double), ("sigma", ctypes.c_double), ("scheme", ctypes.c_int)]


class lbm_batch_params(ctypes.Structure):
    _fields_ = [("tc_mode", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("R", ctypes.c_double), ("G", ctypes.c_double), ("device", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("window", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_steps", ctypes.c_int), ("mode", ctypes.c_int),
                ("rows_per_item", ctypes.c_int), ("conv", ctypes.c_int),
                ("variant", ctypes.c_int), ("conv_rel", ctypes.c_double),
                ("trend_tol", ctypes.c_double)]


class lbm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps", ctypes.c_int), ("rho_g", ctypes.c_double),
                ("rho_l", ctypes.c_double), ("width", ctypes.c_double),
                ("mass", ctypes.c_double), ("max_drho", ctypes.c_double)]


class lbm_batch_stats(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_int), ("launches", ctypes.c_ulonglong),
                ("gpu_ms", ctypes.c_double), ("mode", ctypes.c_int),
                ("rows_per_item", ctypes.c_int), ("n_active", ctypes.c_int)]


(BATCH_AUTO, BATCH_WORKLIST, BATCH_PERSISTENT, BATCH_COOPERATIVE, BATCH_WORKLIST_DYNAMIC,
 BATCH_BALANCED) = range(6)
CONV_COEX, CONV_CELL, CONV_NONE, CONV_TREND = range(4)
RUN_ACTIVE, RUN_CONVERGED, RUN_DIVERGED, RUN_CAPPED = range(4)


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes); the names and order follow include/lbm.h
SIGNATURES = {
    "lbm_default_params": (None, [ctypes.POINTER(lbm_params)]),
    "lbm_create": (_I, [ctypes.POINTER(lbm_params), ctypes.POINTER(_P)]),
    "lbm_init_density": (_I, [_P, _P, _P, _P]),
    "lbm_init_density_at_rest": (_I, [_P, _P]),
    "lbm_create_band": (_I, [_P, _P]),
    "lbm_band_halo_bytes": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_band_halo_pack": (_I, [_P, _P, _P]),
    "lbm_band_halo_unpack": (_I, [_P, _P, _P]),
    "lbm_band_step_overlap": (_I, [_P, _I, _D, _D, _P, _P, _P]),
    "lbm_step": (_I, [_P, _I, _I, _D, _D]),
    "lbm_step_async": (_I, [_P, _I, _I, _D, _D]),
    "lbm_sync_status": (_I, [_P]),
    "lbm_get_moments": (_I, [_P, _P, _P, _P]),
    "lbm_get_mass": (_I, [_P, _DP]),
    "lbm_get_populations": (_I, [_P, _P]),
    "lbm_set_populations": (_I, [_P, _P]),
    "lbm_get_temperature": (_I, [_P, _DP]),
    "lbm_last_error": (ctypes.c_char_p, [_P]),
    "lbm_destroy": (_I, [_P]),
    "lbm_cs_critical_point": (_I, [_D, _D, _D, _DP, _DP, _DP]),
    "lbm_cs_maxwell": (_I, [_D, _D, _D, _D, _DP, _DP, _DP]),
    "lbm_kernel_launch_count": (ctypes.c_ulonglong, []),
    "lbm_set_band_rows": (_I, [_P, _I]),
    "lbm_set_kernel_variant": (_I, [_P, _I]),
    "lbm_get_launch_geometry": (_I, [_P, _I, _IP, _IP, _IP, _IP]),
    "lbm_get_kernel_variant": (_I, [_P, _IP]),
    "lbm_set_mrt_rates": (_I, [_P, _D, _D, _D]),
    "lbm_selftest_wait_timeout": (_I, [_I, ctypes.c_longlong, _IP]),
    "lbm_selftest_grid_barrier_timeout": (_I, [_I, _IP]),
    "lbm_mass_f32_noalloc": (_I, [_P, ctypes.c_size_t, _P, _P]),
    "lbm_host_alloc": (_I, [ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_host_free": (_I, [_P]),
    "lbm_batch_default_params": (None, [ctypes.POINTER(lbm_batch_params)]),
    "lbm_batch_create": (_I, [ctypes.POINTER(lbm_batch_params), ctypes.POINTER(lbm_instance),
                              _I, ctypes.POINTER(_P)]),
    "lbm_batch_init_density": (_I, [_P, _I, _P]),
    "lbm_batch_init_density_at_rest": (_I, [_P, _I, _P]),
    "lbm_batch_init_slabs": (_I, [_P, _P, _P, _P]),
    "lbm_batch_run": (_I, [_P, _I, _IP]),
    "lbm_batch_get_result": (_I, [_P, _I, ctypes.POINTER(lbm_result)]),
    "lbm_batch_get_density": (_I, [_P, _I, _P]),
    "lbm_batch_get_moments": (_I, [_P, _I, _P, _P, _P]),
    "lbm_batch_get_stats": (_I, [_P, ctypes.POINTER(lbm_batch_stats)]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_P]),
    "lbm_batch_destroy": (_I, [_P]),
    "lbm_mlp_num_params": (_I, []),
    "lbm_mlp_create": (_I, [_I, _P, ctypes.POINTER(_P)]),
    "lbm_mlp_destroy": (_I, [_P]),
    "lbm_mlp_last_error": (ctypes.c_char_p, [_P]),
    "lbm_mlp_set_params": (_I, [_P, _P]),
    "lbm_mlp_get_params": (_I, [_P, _P]),
    "lbm_mlp_gradient": (_I, [_P, _P, _P, _I, _P, _P]),
    "lbm_mlp_train": (_I, [_P, _P, _P, _I, _P, _I, _I, ctypes.c_float, _P]),
    "lbm_mlp_predict": (_I, [_P, _P, _I, _P]),
}

_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _fwd(name):
    def call(*args):
        return getattr(lib(), name)(*args)
    call.__name__ = name
    return call


for _name in SIGNATURES:
    globals()[_name] = _fwd(_name)


def _dptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(int(a))  # a raw pointer (e.g. pinned torch memory)


def host_array(shape, dtype=np.float64):
    """Zeroed numpy array in page-locked host memory from lbm_host_alloc (huge
    pages where the kernel provides them), for the host arrays the C ABI
    copies; the memory goes back through lbm_host_free when the array (and
    every view of it) is collected."""
    dtype = np.dtype(dtype)
    count = int(np.prod(shape))
    nbytes = max(count * dtype.itemsize, 1)
    p = ctypes.c_void_p()
    st = lib().lbm_host_alloc(nbytes, ctypes.byref(p))
    if st != LBM_OK:
        raise LbmError(st, "lbm_host_alloc failed")
    buf = (ctypes.c_char * nbytes).from_address(p.value)
    arr = np.frombuffer(buf, dtype=dtype, count=count).reshape(shape)
    weakref.finalize(buf, lib().lbm_host_free, ctypes.c_void_p(p.value))
    return arr


def critical_point(a=1.0, b=4.0, R=1.0):
    rc, tc, pc = _D(), _D(), _D()
    st = lib().lbm_cs_critical_point(a, b, R, ctypes.byref(rc), ctypes.byref(tc), ctypes.byref(pc))
    if st:
        raise LbmError(st, "lbm_cs_critical_point")
    return rc.value, tc.value, pc.value


def maxwell(T, a=1.0, b=4.0, R=1.0):
    """(rho_g, rho_l, p0) of the Maxwell construction at absolute T."""
    rg, rl, p0 = _D(), _D(), _D()
    st = lib().lbm_cs_maxwell(T, a, b, R, ctypes.byref(rg), ctypes.byref(rl), ctypes.byref(p0))
    if st:
        raise LbmError(st, "lbm_cs_maxwell")
    return rg.value, rl.value, p0.value


def temperature(T_over_Tc, tc_mode=0, a=1.0, b=4.0, R=1.0):
    return T_over_Tc * (critical_point(a, b, R)[1] if tc_mode == 0 else 0.094)


def selftest_wait_timeout(device=0, polls=1000):
    """Status of a bounded device wait that nothing completes (LBM_E_TIMEOUT
    expected); raises on bad arguments or CUDA errors."""
    r = _I()
    st = lib().lbm_selftest_wait_timeout(int(device), int(polls), ctypes.byref(r))
    if st:
        raise LbmError(st, "lbm_selftest_wait_timeout")
    return r.value


def selftest_grid_barrier_timeout(device=0):
    """Status of the batch grid barrier when one CTA never arrives
    (LBM_E_TIMEOUT expected)."""
    r = _I()
    st = lib().lbm_selftest_grid_barrier_timeout(int(device), ctypes.byref(r))
    if st:
        raise LbmError(st, "lbm_selftest_grid_barrier_timeout")
    return r.value


def launch_count():
    return int(lib().lbm_kernel_launch_count())


class Lattice:
    """A context of the C ABI with numpy in/out (same life cycle as lbm_*)."""

    def __init__(self, nx, ny, T_over_Tc, precision=FP32, tc_mode=0, a=1.0, b=4.0,
                 R=1.0, G=-1.0, device=0, stream=None, band=False):
        """band=True: ny rows of a y-decomposed lattice (lbm_create_band); its
        initial densities then have ny + 4 rows (two halo rows each side)."""
        p = lbm_params()
        lib().lbm_default_params(ctypes.byref(p))
        p.nx, p.ny, p.T_over_Tc, p.tc_mode = int(nx), int(ny), float(T_over_Tc), int(tc_mode)
        p.a, p.b, p.R, p.G = a, b, R, G
        p.precision, p.device = int(precision), int(device)
        p.cuda_stream = None if stream is None else ctypes.c_void_p(int(stream))
        ctx = _P()
        create = lib().lbm_create_band if band else lib().lbm_create
        st = create(ctypes.byref(p), ctypes.byref(ctx))
        if st:
            raise LbmError(st, lib().lbm_last_error(None).decode())
        self.ctx = ctx
        self.nx, self.ny = int(nx), int(ny)
        self.precision = precision
        self.band = bool(band)
        self.init_rows = self.ny + 4 if band else self.ny

    def halo_bytes(self):
        n = ctypes.c_size_t()
        self._check(lib().lbm_band_halo_bytes(self.ctx, ctypes.byref(n)), "lbm_band_halo_bytes")
        return n.value

    def halo_pack(self, d_lo, d_hi):
        """Queue the copies of the two lowest / highest owned rows into the
        device buffers at addresses d_lo, d_hi."""
        self._check(lib().lbm_band_halo_pack(self.ctx, _P(int(d_lo)), _P(int(d_hi))),
                    "lbm_band_halo_pack")

    def step_overlap(self, scheme, tau, sigma, d_lo, d_hi, comm_stream=None):
        """One band step with the boundary rows first, packed into d_lo /
        d_hi, and comm_stream made to wait for the pack (lbm_band_step_overlap)."""
        self._check(lib().lbm_band_step_overlap(
            self.ctx, int(scheme), float(tau), float(sigma), _P(int(d_lo)), _P(int(d_hi)),
            None if comm_stream is None else _P(int(comm_stream))), "lbm_band_step_overlap")

    def halo_unpack(self, d_below, d_above):
        self._check(lib().lbm_band_halo_unpack(self.ctx, _P(int(d_below)), _P(int(d_above))),
                    "lbm_band_halo_unpack")

    def _check(self, st, what):
        if st:
            raise LbmError(st, f"{what}: {lib().lbm_last_error(self.ctx).decode()}")

    def close(self):
        if self.ctx:
            lib().lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def T(self):
        t = _D()
        self._check(lib().lbm_get_temperature(self.ctx, ctypes.byref(t)), "lbm_get_temperature")
        return t.value

    def init_density(self, rho, ux=None, uy=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        ux = None if ux is None else np.ascontiguousarray(ux, dtype=np.float64)
        uy = None if uy is None else np.ascontiguousarray(uy, dtype=np.float64)
        assert rho.shape == (self.init_rows, self.nx)
        self._check(lib().lbm_init_density(self.ctx, _dptr(rho), _dptr(ux), _dptr(uy)),
                    "lbm_init_density")

    def init_density_at_rest(self, rho):
        """f = f_eq(rho, u) with u = -F / (2 rho): zero actual velocity."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        assert rho.shape == (self.init_rows, self.nx)
        self._check(lib().lbm_init_density_at_rest(self.ctx, _dptr(rho)),
                    "lbm_init_density_at_rest")

    def step(self, n, scheme, tau, sigma=0.0, raise_on_error=True):
        st = lib().lbm_step(self.ctx, int(n), int(scheme), float(tau), float(sigma))
        if raise_on_error:
            self._check(st, "lbm_step")
        return st

    def step_async(self, n, scheme, tau, sigma=0.0):
        self._check(lib().lbm_step_async(self.ctx, int(n), int(scheme), float(tau),
                                         float(sigma)), "lbm_step_async")

    def sync(self):
        return lib().lbm_sync_status(self.ctx)

    def observe(self, out=None):
        """(rho, vx, vy) as FP64 arrays; `out` may supply the three arrays
        (host_array buffers keep the copies at the link rate)."""
        if out is None:
            out = tuple(np.empty((self.ny, self.nx)) for _ in range(3))
        rho, vx, vy = out
        self._check(lib().lbm_get_moments(self.ctx, _dptr(rho), _dptr(vx), _dptr(vy)),
                    "lbm_get_moments")
        return rho, vx, vy

    def mass(self):
        m = _D()
        self._check(lib().lbm_get_mass(self.ctx, ctypes.byref(m)), "lbm_get_mass")
        return m.value

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        self._check(lib().lbm_get_populations(self.ctx, _dptr(f)), "lbm_get_populations")
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx)
        self._check(lib().lbm_set_populations(self.ctx, _dptr(f)), "lbm_set_populations")

    def set_variant(self, variant):
        self._check(lib().lbm_set_kernel_variant(self.ctx, int(variant)),
                    "lbm_set_kernel_variant")

    def set_band_rows(self, rows):
        self._check(lib().lbm_set_band_rows(self.ctx, int(rows)), "lbm_set_band_rows")

    def geometry(self, scheme=SC):
        v = [_I() for _ in range(4)]
        self._check(lib().lbm_get_launch_geometry(self.ctx, int(scheme),
                                                  *[ctypes.byref(x) for x in v]),
                    "lbm_get_launch_geometry")
        return dict(zip(("n_strips", "band_rows", "n_bands", "grid"), (x.value for x in v)))

    def set_mrt_rates(self, s_e=0.0, s_eps=0.0, s_q=0.0):
        """Rates of the MRT scheme's energy, energy-square and energy-flux
        moments (<= 0: 1/tau)."""
        self._check(lib().lbm_set_mrt_rates(self.ctx, float(s_e), float(s_eps), float(s_q)),
                    "lbm_set_mrt_rates")

    def variant(self):
        """The kernel variant lbm_step resolves to (VARIANT_REGISTER/STAGED/PAIR)."""
        v = _I()
        self._check(lib().lbm_get_kernel_variant(self.ctx, ctypes.byref(v)),
                    "lbm_get_kernel_variant")
        return v.value


class Batch:
    """A batch of independent instances (lbm_batch_* of the C ABI).

    `instances` is a list of dicts with nx, ny, T_over_Tc, tau, sigma, scheme.
    """

    def __init__(self, instances, window=1000, tol=1e-9, max_steps=200000, mode=BATCH_AUTO,
                 rows_per_item=0, tc_mode=0, device=0, stream=None, conv=CONV_COEX,
                 variant=VARIANT_AUTO, conv_rel=None, trend_tol=None):
        p = lbm_batch_params()
        lib().lbm_batch_default_params(ctypes.byref(p))
        p.window, p.tol, p.max_steps, p.conv = int(window), float(tol), int(max_steps), int(conv)
        p.variant = int(variant)
        if conv_rel is not None:
            p.conv_rel = float(conv_rel)
        if trend_tol is not None:
            p.trend_tol = float(trend_tol)
        p.mode, p.rows_per_item, p.tc_mode, p.device = int(mode), int(rows_per_item), \
            int(tc_mode), int(device)
        p.cuda_stream = None if stream is None else ctypes.c_void_p(int(stream))
        arr = (lbm_instance * len(instances))()
        for k, d in enumerate(instances):
            arr[k] = lbm_instance(int(d["nx"]), int(d["ny"]), float(d["T_over_Tc"]),
                                  float(d["tau"]), float(d.get("sigma", 0.0)),
                                  int(d["scheme"]))
        h = _P()
        st = lib().lbm_batch_create(ctypes.byref(p), arr, len(instances), ctypes.byref(h))
        if st:
            raise LbmError(st, "lbm_batch_create")
        self.h = h
        self.instances = [dict(d) for d in instances]

    def _check(self, st, what):
        if st:
            raise LbmError(st, f"{what}: {lib().lbm_batch_last_error(self.h).decode()}")

    def close(self):
        if self.h:
            lib().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return len(self.instances)

    def init_density(self, i, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        d = self.instances[i]
        assert rho.shape == (d["ny"], d["nx"])
        self._check(lib().lbm_batch_init_density(self.h, int(i), _dptr(rho)),
                    "lbm_batch_init_density")

    def init_density_at_rest(self, i, rho):
        """Instance i from rho at zero actual velocity (u = -F / (2 rho))."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        d = self.instances[i]
        assert rho.shape == (d["ny"], d["nx"])
        self._check(lib().lbm_batch_init_density_at_rest(self.h, int(i), _dptr(rho)),
                    "lbm_batch_init_density_at_rest")

    def init_slabs(self, rho_g, rho_l, width):
        g, l, w = (np.ascontiguousarray(v, dtype=np.float64) for v in (rho_g, rho_l, width))
        assert len(g) == len(l) == len(w) == len(self)
        self._check(lib().lbm_batch_init_slabs(self.h, _dptr(g), _dptr(l), _dptr(w)),
                    "lbm_batch_init_slabs")

    def run(self, max_windows=1 << 30):
        n = _I()
        self._check(lib().lbm_batch_run(self.h, int(max_windows), ctypes.byref(n)),
                    "lbm_batch_run")
        return n.value

    def result(self, i):
        r = lbm_result()
        self._check(lib().lbm_batch_get_result(self.h, int(i), ctypes.byref(r)),
                    "lbm_batch_get_result")
        return {k: getattr(r, k) for k, _ in lbm_result._fields_}

    def results(self):
        return [self.result(i) for i in range(len(self))]

    def density(self, i):
        d = self.instances[i]
        rho = np.empty((d["ny"], d["nx"]))
        self._check(lib().lbm_batch_get_density(self.h, int(i), _dptr(rho)),
                    "lbm_batch_get_density")
        return rho

    def moments(self, i):
        """(rho, vx, vy) of instance i; v is the actual velocity u + F/(2 rho)."""
        d = self.instances[i]
        out = [np.empty((d["ny"], d["nx"])) for _ in range(3)]
        self._check(lib().lbm_batch_get_moments(self.h, int(i), *[_dptr(a) for a in out]),
                    "lbm_batch_get_moments")
        return tuple(out)

    def stats(self):
        s = lbm_batch_stats()
        self._check(lib().lbm_batch_get_stats(self.h, ctypes.byref(s)), "lbm_batch_get_stats")
        return {k: getattr(s, k) for k, _ in lbm_batch_stats._fields_}


def _fptr(a, dtype=np.float32):
    assert a.dtype == dtype and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


class MLP:
    """The warm-start network of the C ABI (lbm_mlp_*), FP32."""

    def __init__(self, params=None, device=0, stream=None):
        h = _P()
        st = lib().lbm_mlp_create(int(device), None if stream is None else
                                  ctypes.c_void_p(int(stream)), ctypes.byref(h))
        if st:
            raise LbmError(st, "lbm_mlp_create")
        self.h = h
        self.n_params = int(lib().lbm_mlp_num_params())
        if params is not None:
            self.set_params(params)

    def _check(self, st, what):
        if st:
            raise LbmError(st, f"{what}: {lib().lbm_mlp_last_error(self.h).decode()}")

    def close(self):
        if self.h:
            lib().lbm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.shape == (self.n_params,)
        self._check(lib().lbm_mlp_set_params(self.h, _fptr(p)), "lbm_mlp_set_params")

    def params(self):
        p = np.empty(self.n_params, dtype=np.float32)
        self._check(lib().lbm_mlp_get_params(self.h, _fptr(p)), "lbm_mlp_get_params")
        return p

    def gradient(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        self._check(lib().lbm_mlp_gradient(self.h, _fptr(X), _fptr(Y), len(X), _fptr(g),
                                           _fptr(loss)), "lbm_mlp_gradient")
        return float(loss[0]), g

    def train(self, X, Y, order, batch, lr):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        order = np.ascontiguousarray(order, dtype=np.int32)
        loss = np.zeros(1, dtype=np.float32)
        self._check(lib().lbm_mlp_train(self.h, _fptr(X), _fptr(Y), len(X),
                                        _fptr(order, np.int32), order.shape[0], int(batch),
                                        float(lr), _fptr(loss)), "lbm_mlp_train")
        return float(loss[0])

    def predict(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.empty((len(X), 3), dtype=np.float32)
        self._check(lib().lbm_mlp_predict(self.h, _fptr(X), len(X), _fptr(Y)),
                    "lbm_mlp_predict")
        return Y
