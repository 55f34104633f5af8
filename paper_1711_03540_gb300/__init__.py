"""Python binding of the GB300 lattice Boltzmann library for the
Kuramoto-Sivashinsky equation (arXiv:1711.03540).

Argument marshalling only: every function here has the name of, and calls,
one entry point of the C ABI declared in ``include/lb_ks.h``; all the work
happens in the CUDA library ``liblbks.so`` built in-tree by ``build.py``.
There is no fallback: importing works without the library, but the first
call raises if ``liblbks.so`` is missing.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
they must be contiguous.  ``LbKsOpts.stream`` accepts a ``torch.cuda.Stream``
or a raw ``cudaStream_t`` integer.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = [
    "LbKsError", "LbKsOpts", "lb_ks_default_opts", "lb_ks_params", "lb_ks_tau_fit", "lb_ks_init",
    "lb_ks_batch_init", "lb_ks_batch_init_reservoir", "lb_ks_step", "lb_ks_rho", "lb_ks_mass_energy", "lb_ks_state_bytes", "lb_ks_save",
    "lb_ks_load", "lb_ks_steps_done", "lb_ks_describe", "lb_ks_launches", "lb_ks_fma_peak",
    "lb_ks_mass_energy_noalloc", "lb_ks_set_link_test", "lb_ks_free",
    "lb_ks_last_error", "library_path", "D1Q5", "D1Q7", "F64", "F32", "F16S", "KERNEL_AUTO", "KERNEL_PLAIN",
    "KERNEL_STREAM", "KERNEL_RESIDENT", "ABI_FUNCTIONS",
]

D1Q5, D1Q7 = 5, 7
F64, F32, F16S = 0, 1, 2
KERNEL_AUTO, KERNEL_PLAIN, KERNEL_STREAM, KERNEL_RESIDENT, KERNEL_COLLAPSE = 0, 1, 2, 3, 4
DM_DERIVED, DM_PRINTED = 0, 1
WEIGHTS_FULL_INVERSE = 2  # flag: D1Q7 with the full 7-speed inverse weights (an ablation)
STATUS = {0: "LB_KS_OK", -1: "LB_KS_EINVAL", -2: "LB_KS_ENOMEM", -3: "LB_KS_ECUDA", -4: "LB_KS_EUNSTABLE",
          -5: "LB_KS_ETIMEOUT"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liblbks.so")
_lock = threading.Lock()
_lib = None


class LbKsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class LbKsOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("dm_variant", C.c_int32), ("recentre_every", C.c_int32),
                ("kernel", C.c_int32), ("steps_per_launch", C.c_int32), ("sites_per_thread", C.c_int32),
                ("threads_per_block", C.c_int32), ("use_graph", C.c_int32), ("autotune", C.c_int32),
                ("stream", C.c_void_p), ("cluster_size", C.c_int32)]


_P = C.c_void_p
_PD = C.POINTER(C.c_double)
# name -> (restype, argtypes): the C ABI of include/lb_ks.h
ABI_FUNCTIONS = {
    "lb_ks_default_opts": (None, [C.POINTER(LbKsOpts)]),
    "lb_ks_params": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, _PD, _PD, _PD]),
    "lb_ks_tau_fit": (C.c_double, [C.c_int, C.c_double, C.c_double]),
    "lb_ks_max_growth": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int, _PD]),
    "lb_ks_init": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int64, C.c_double, C.c_double, C.c_double, _P,
                             C.POINTER(LbKsOpts)]),
    "lb_ks_batch_init": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int32, _P, _P, _P, _P, _P, C.POINTER(LbKsOpts)]),
    "lb_ks_batch_init_reservoir": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int32, _P, _P, _P, _P, _P, _P, _P,
                                             C.POINTER(LbKsOpts)]),
    "lb_ks_step": (C.c_int, [_P, C.c_int64]),
    "lb_ks_rho": (C.c_int, [_P, _P]),
    "lb_ks_mass_energy": (C.c_int, [_P, _P, _P]),
    "lb_ks_state_bytes": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "lb_ks_save": (C.c_int, [_P, _P, C.c_size_t]),
    "lb_ks_load": (C.c_int, [_P, _P, C.c_size_t]),
    "lb_ks_steps_done": (C.c_int64, [_P]),
    "lb_ks_describe": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "lb_ks_describe_lanes": (C.c_int, [_P, C.POINTER(C.c_int32), C.c_int]),
    "lb_ks_launches": (C.c_int64, [_P]),
    "lb_ks_fma_peak": (C.c_int, [C.c_int, _PD]),
    "lb_ks_mass_energy_noalloc": (C.c_int, [C.c_int, C.c_int, _P, C.c_int64, C.c_int64, C.c_double, C.c_double, _P,
                                            _P]),
    "lb_ks_set_link_test": (C.c_int, [_P, C.c_int32, C.c_uint32]),
    "lb_ks_free": (None, [_P]),
    "lb_ks_last_error": (C.c_char_p, [_P]),
}


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'` (CUDA path only, no fallback)")
            lib = C.CDLL(_LIB_PATH)
            for name, (res, args) in ABI_FUNCTIONS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int, h=None):
    if rc != 0:
        raise LbKsError(rc, lb_ks_last_error(h))


def _ptr(a, dtype=np.float64):
    """Data pointer of a contiguous numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if (dtype is not None and a.dtype != dtype) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"expected a contiguous {np.dtype(dtype).name} array")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)!r}")


def lb_ks_default_opts(**kw) -> LbKsOpts:
    o = LbKsOpts()
    _load().lb_ks_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "stream":
            v = getattr(v, "cuda_stream", v)
            o.stream = C.c_void_p(int(v) if v else 0)
        else:
            setattr(o, k, int(v))
    return o


def lb_ks_params(scheme: int, dx: float, dt: float, tau: float, dm_variant: int = DM_DERIVED):
    """Returns (A, B, coef) with f^eq_i = A_i rho + B_i rho^2 and coef = (T1..T4, J, K, M, dM, E)."""
    A = np.zeros(scheme)
    B = np.zeros(scheme)
    coef = np.zeros(9)
    rc = _load().lb_ks_params(scheme, dx, dt, tau, dm_variant, A.ctypes.data_as(_PD), B.ctypes.data_as(_PD),
                              coef.ctypes.data_as(_PD))
    if rc != 0:
        raise LbKsError(rc, "invalid parameters")
    return A, B, coef


def lb_ks_tau_fit(scheme: int, dX: float, dT: float) -> float:
    return float(_load().lb_ks_tau_fit(scheme, dX, dT))


def lb_ks_max_growth(scheme: int, dx: float, dt: float, tau: float, dm_variant: int = DM_DERIVED,
                     rho_bar: float = 0.0, nk: int = 256) -> float:
    """Largest linear growth rate per unit time over all branches and nk phases."""
    g = C.c_double(0.0)
    _check(_load().lb_ks_max_growth(scheme, dx, dt, tau, dm_variant, rho_bar, nk, C.byref(g)))
    return g.value


def lb_ks_init(scheme: int, N: int, L: float, dt: float, tau: float, rho0, opts: LbKsOpts | None = None):
    h = C.c_void_p()
    rc = _load().lb_ks_init(C.byref(h), scheme, int(N), float(L), float(dt), float(tau), _ptr(rho0),
                            C.byref(opts) if opts is not None else None)
    _check(rc)
    return h


def lb_ks_batch_init(scheme: int, N, L, dt, tau, rho0, opts: LbKsOpts | None = None):
    N = np.ascontiguousarray(N, dtype=np.int64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    h = C.c_void_p()
    rc = _load().lb_ks_batch_init(C.byref(h), scheme, len(N), _ptr(N, np.int64), _ptr(L), _ptr(dt), _ptr(tau),
                                  _ptr(rho0), C.byref(opts) if opts is not None else None)
    _check(rc)
    return h


def lb_ks_batch_init_reservoir(scheme: int, N, L, dt, tau, rho0, rho_left, rho_right, opts: LbKsOpts | None = None):
    N = np.ascontiguousarray(N, dtype=np.int64)
    L, dt, tau, rl, rr = (np.ascontiguousarray(v, dtype=np.float64) for v in (L, dt, tau, rho_left, rho_right))
    h = C.c_void_p()
    rc = _load().lb_ks_batch_init_reservoir(C.byref(h), scheme, len(N), _ptr(N, np.int64), _ptr(L), _ptr(dt),
                                            _ptr(tau), _ptr(rho0), _ptr(rl), _ptr(rr),
                                            C.byref(opts) if opts is not None else None)
    _check(rc)
    return h


def lb_ks_step(h, n: int) -> None:
    _check(_load().lb_ks_step(h, int(n)), h)


def lb_ks_rho(h, out) -> None:
    _check(_load().lb_ks_rho(h, _ptr(out)), h)


def lb_ks_mass_energy(h, mass, energy) -> None:
    _check(_load().lb_ks_mass_energy(h, _ptr(mass), _ptr(energy)), h)


def lb_ks_state_bytes(h) -> int:
    n = C.c_size_t(0)
    _check(_load().lb_ks_state_bytes(h, C.byref(n)), h)
    return n.value


def lb_ks_save(h, buf: np.ndarray) -> None:
    _check(_load().lb_ks_save(h, _ptr(buf, np.uint8), buf.nbytes), h)


def lb_ks_load(h, buf: np.ndarray) -> None:
    _check(_load().lb_ks_load(h, _ptr(buf, np.uint8), buf.nbytes), h)


def lb_ks_steps_done(h) -> int:
    return int(_load().lb_ks_steps_done(h))


def lb_ks_describe(h) -> dict:
    k, s, t, l, cl = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
    nr, tot = C.c_int32(), C.c_int64()
    _check(_load().lb_ks_describe(h, C.byref(k), C.byref(s), C.byref(t), C.byref(l), C.byref(cl), C.byref(nr),
                                  C.byref(tot)), h)
    return {"kernel": k.value, "sites_per_thread": s.value, "threads_per_block": t.value,
            "steps_per_launch": l.value, "cluster_size": cl.value, "nruns": nr.value, "total_sites": tot.value}


LANE_FIELDS = ("blocks_per_group", "groups", "bundles", "steps_per_launch", "segmented", "pair_exchange_steps",
               "merged_single_blocks", "halved_lattices")


def lb_ks_describe_lanes(h) -> list:
    """The resident plan: one dict per concurrent lane (empty when not resident)."""
    buf = (C.c_int32 * (8 * len(LANE_FIELDS)))()
    n = _load().lb_ks_describe_lanes(h, buf, 8)
    if n < 0:
        _check(n, h)
    return [dict(zip(LANE_FIELDS, buf[len(LANE_FIELDS) * l:len(LANE_FIELDS) * (l + 1)])) for l in range(min(n, 8))]


def lb_ks_launches(h) -> int:
    return int(_load().lb_ks_launches(h))


def lb_ks_fma_peak(fp64: bool) -> float:
    v = C.c_double(0.0)
    rc = _load().lb_ks_fma_peak(int(bool(fp64)), C.byref(v))
    _check(rc)
    return v.value


def lb_ks_mass_energy_noalloc(scheme: int, precision: int, f, plane: int, N: int, rhobar: float, scale: float,
                              out, stream=None) -> None:
    """Mass and energy of populations held by the caller (device memory), with no allocation."""
    s = getattr(stream, "cuda_stream", stream)
    rc = _load().lb_ks_mass_energy_noalloc(scheme, precision, _ptr(f, None), int(plane), int(N), float(rhobar),
                                           float(scale), _ptr(out), C.c_void_p(int(s) if s else 0))
    _check(rc)


def lb_ks_set_link_test(h, withhold_step: int, wait_rounds: int = 0) -> None:
    """Testing aid: withhold block 1's sends across a cluster pair's edge at one step."""
    _check(_load().lb_ks_set_link_test(h, int(withhold_step), int(wait_rounds)), h)


def lb_ks_free(h) -> None:
    if h:
        _load().lb_ks_free(h)


def lb_ks_last_error(h=None) -> str:
    s = _load().lb_ks_last_error(h)
    return s.decode() if s else ""
