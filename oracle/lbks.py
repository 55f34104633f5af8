"""ctypes front end of the plain FP64 C oracle (``lbks_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  ``build()`` compiles
the C file with gcc; ``load()`` returns the library, building it on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbks_oracle.c")
_LIB = os.path.join(_HERE, "liblbks_oracle.so")
_lock = threading.Lock()
_lib = None

D1Q5, D1Q7 = 5, 7
DM_DERIVED, DM_PRINTED = 0, 1
WEIGHTS_FULL_INVERSE = 2  # flag (D1Q7): w1, w2, w4 of the full 7-speed inverse, an ablation


def build(force: bool = False) -> str:
    """Compile ``lbks_oracle.c`` into ``liblbks_oracle.so`` (plain -O2, no FMA
    contraction so that rounding is the same on x86 and Arm)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _LIB


def load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            d, i64, i32 = C.c_double, C.c_int64, C.c_int
            pd = C.POINTER(C.c_double)
            lib.lbo_coefficients.argtypes = [i32, d, d, d, i32, pd]
            lib.lbo_weight.argtypes = [i32, i32, i32, pd]
            lib.lbo_weight_full.argtypes = [i32, i32, pd]
            lib.lbo_speed.argtypes = [i32, i32]
            lib.lbo_feq.argtypes = [i32, d, d, d, i32, i32, d, pd]
            lib.lbo_run.argtypes = [i32, i64, d, d, d, i32, i32, i32, d, d, pd, i64, pd, pd]
            lib.lbo_run_batch.argtypes = [i32, C.c_int32, C.POINTER(C.c_int64), pd, pd, pd, i32,
                                          pd, i64, pd, i32, C.POINTER(C.c_int)]
            lib.lbo_set_mutation.argtypes = [i32]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def speeds(Q: int) -> np.ndarray:
    lib = load()
    return np.array([lib.lbo_speed(Q, i) for i in range(Q)], dtype=np.int64)


def weight(Q: int, l: int) -> np.ndarray:
    """w^(l)_i over the Q speeds, as the oracle uses them."""
    lib = load()
    out = np.empty(Q)
    v = C.c_double()
    for i in range(Q):
        if lib.lbo_weight(Q, l, i, C.byref(v)) != 0:
            raise ValueError(f"no weight w^({l}) for Q={Q}")
        out[i] = v.value
    return out


def weight_full(l: int) -> np.ndarray:
    """w^(l)_i of the full 7-speed inverse of Appendix A's moment matrix."""
    lib = load()
    out = np.empty(7)
    for i in range(7):
        w = C.c_double()
        if lib.lbo_weight_full(l, i, C.byref(w)) != 0:
            raise ValueError("bad weight index")
        out[i] = w.value
    return out


def coefficients(Q: int, alpha: float, beta: float, tau: float, dm_variant: int = DM_DERIVED) -> dict:
    """T1..T4 (Eq. T_form), J, K, M (Table 2), delta M (Eq. delta_M), E (delta f^eq)."""
    out = np.zeros(9)
    rc = load().lbo_coefficients(Q, alpha, beta, tau, dm_variant, _p(out))
    if rc != 0:
        raise ValueError("invalid parameters")
    keys = ["T1", "T2", "T3", "T4", "J", "K", "M", "dM", "E"]
    return dict(zip(keys, out.tolist()))


def feq(Q: int, alpha: float, beta: float, tau: float, rho: float, dm_variant: int = DM_DERIVED,
        advection: bool = True) -> np.ndarray:
    out = np.zeros(Q)
    rc = load().lbo_feq(Q, alpha, beta, tau, dm_variant, int(advection), rho, _p(out))
    if rc != 0:
        raise ValueError("invalid parameters")
    return out


def feq_linear_quadratic(Q, alpha, beta, tau, dm_variant=DM_DERIVED, advection=True):
    """(A, B) with f^eq_i(rho) = A_i rho + B_i rho^2, read off the oracle's own
    equilibrium at rho = +1 and -1 (exact: f^eq is a quadratic in rho)."""
    fp = feq(Q, alpha, beta, tau, 1.0, dm_variant, advection)
    fm = feq(Q, alpha, beta, tau, -1.0, dm_variant, advection)
    return 0.5 * (fp - fm), 0.5 * (fp + fm)


def run(Q: int, rho0, alpha: float, beta: float, tau: float, nsteps: int, *, dm_variant: int = DM_DERIVED,
        advection: bool = True, boundary: str = "periodic", rho_left: float = 0.0, rho_right: float = 0.0,
        return_f: bool = False):
    """Run the LB scheme from f = f^eq(rho0) for nsteps steps; return rho (and f[Q, N])."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    N = rho0.shape[0]
    rho = np.empty(N)
    f = np.empty((Q, N)) if return_f else None
    bnd = {"periodic": 0, "reservoir": 1}[boundary]
    rc = load().lbo_run(Q, N, alpha, beta, tau, dm_variant, int(advection), bnd, rho_left, rho_right,
                        _p(rho0), int(nsteps), _p(rho), _p(f) if f is not None else None)
    if rc != 0:
        raise ValueError(f"oracle run failed ({rc})")
    return (rho, f) if return_f else rho


def run_batch(Q: int, N, alpha, beta, tau, rho0, nsteps: int, *, dm_variant: int = DM_DERIVED,
              nthreads: int = 1):
    """Independent periodic runs; rho0 concatenated in run order.  Returns (rho, threads used)."""
    N = np.ascontiguousarray(N, dtype=np.int64)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    out = np.empty_like(rho0)
    used = C.c_int(0)
    rc = load().lbo_run_batch(Q, len(N), N.ctypes.data_as(C.POINTER(C.c_int64)), _p(alpha), _p(beta), _p(tau),
                              dm_variant, _p(rho0), int(nsteps), _p(out), int(nthreads), C.byref(used))
    if rc != 0:
        raise ValueError(f"oracle batch failed ({rc})")
    return out, used.value


class mutation:
    """Context manager that plants a deliberate mistake in the oracle (tests only).
    1 flips the streaming direction, 3 drops K w2, 4 flips the sign of J, 5 drops delta f^eq."""

    def __init__(self, m: int):
        self.m = m

    def __enter__(self):
        load().lbo_set_mutation(self.m)
        return self

    def __exit__(self, *exc):
        load().lbo_set_mutation(0)
        return False
