"""Analytic travelling-front solution of the KS equation (Table 5) and the
global relative error G (Sec. 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

B = 3.0  # b
X_MIN, X_MAX = 0.0, 60.0  # X_m, X_M
X0 = (X_MAX - X_MIN) / 3.0
KW = 0.5 * np.sqrt(11.0 / 19.0)  # k of Table 5
AMP = 15.0 / 19.0 * np.sqrt(11.0 / 19.0)


def rho_exact(X, T):
    """Table 5, analytic solution: b + (15/19) sqrt(11/19) {-9 tanh z + 11 tanh^3 z},
    z = k (X - b T - X0)."""
    z = np.tanh(KW * (np.asarray(X, dtype=np.float64) - B * T - X0))
    return B + AMP * (-9.0 * z + 11.0 * z ** 3)


RHO_LEFT = B - 30.0 / 19.0 * np.sqrt(11.0 / 19.0)  # Table 5, rho(X_m, t)
RHO_RIGHT = 2.0 * B - RHO_LEFT  # Table 5, rho(X_M, t)


def global_relative_error(rho_num, rho_ref) -> float:
    """G of Sec. 3: sum |rho^N - rho^A| / sum |rho^A|."""
    rho_num = np.asarray(rho_num)
    rho_ref = np.asarray(rho_ref)
    return float(np.sum(np.abs(rho_num - rho_ref)) / np.sum(np.abs(rho_ref)))


def nodes(alpha: float) -> np.ndarray:
    n = int(round((X_MAX - X_MIN) / alpha)) + 1
    return X_MIN + alpha * np.arange(n)
