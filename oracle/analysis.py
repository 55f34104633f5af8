"""Linear analysis of one LB step: amplification matrix, growth rates,
truncation-error predictions of Sec. 2.2, linear stability scans.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Linearising f^eq_i(rho) = A_i rho + B_i rho^2 about a uniform state rho_bar
gives a_i = A_i + 2 B_i rho_bar.  For a Fourier mode f_i(x, t) = fhat_i(t)
exp(i kappa x) the step of Eq. LB_equation_ordinary (collide, then
f_i(x + c_i) <- f*_i(x)) is fhat(t+1) = G(kappa) fhat(t) with

    G(kappa) = diag(exp(-i kappa c_i)) ((1 - 1/tau) I + (1/tau) a 1^T).

A and B are read off the C oracle's own equilibrium (lbks.feq_linear_quadratic),
so these tools test that code, not a second transcription of the paper.
"""
from __future__ import annotations

import math

import numpy as np

from . import lbks


def t_series(i: int, tau: float, nmax: int = 20000) -> float:
    """T_i by its defining series, Sec. 2 (below Eq. feq):
    sum_{n>=1} (1 - 1/tau)^n [(n+1)^i - n^i].  Plain summation in float64."""
    q = 1.0 - 1.0 / tau
    s = 0.0
    term_q = 1.0
    for n in range(1, nmax + 1):
        term_q *= q
        if term_q == 0.0:
            break
        s += term_q * ((n + 1) ** i - n ** i)
    return s


def amplification_matrix(Q: int, a: np.ndarray, tau: float, kappa: float) -> np.ndarray:
    c = lbks.speeds(Q)
    r = 1.0 - 1.0 / tau
    w = 1.0 / tau
    inner = r * np.eye(Q) + w * np.outer(a, np.ones(Q))
    return np.diag(np.exp(-1j * kappa * c)) @ inner


def linearised_a(Q, alpha, beta, tau, rho_bar=0.0, dm_variant=lbks.DM_DERIVED, advection=True):
    A, B = lbks.feq_linear_quadratic(Q, alpha, beta, tau, dm_variant, advection)
    return A + 2.0 * B * rho_bar


def hydro_eigenvalue(Q, alpha, beta, tau, k, rho_bar=0.0, dm_variant=lbks.DM_DERIVED, precise=False):
    """Eigenvalue of G(k alpha) on the hydrodynamic branch (the one that tends
    to 1 as k -> 0), for physical wavenumber k.  ``precise`` uses mpmath at 40
    digits (the growth-rate error terms are ~1e-8 of the eigenvalue)."""
    a = linearised_a(Q, alpha, beta, tau, rho_bar, dm_variant)
    kappa = k * alpha
    if not precise:
        lam = np.linalg.eigvals(amplification_matrix(Q, a, tau, kappa))
        return complex(lam[np.argmin(np.abs(lam - 1.0))])
    import mpmath as mp

    mp.mp.dps = 40
    c = lbks.speeds(Q)
    r = 1 - mp.mpf(1) / mp.mpf(tau)
    w = mp.mpf(1) / mp.mpf(tau)
    G = mp.matrix(Q, Q)
    for i in range(Q):
        ph = mp.exp(-1j * mp.mpf(kappa) * int(c[i]))
        for j in range(Q):
            G[i, j] = ph * ((r if i == j else 0) + w * mp.mpf(a[i]))
    ev = mp.eig(G, left=False, right=False)
    best = min(ev, key=lambda z: abs(z - 1))
    return complex(best)


def growth_rate(Q, alpha, beta, tau, k, dm_variant=lbks.DM_DERIVED, precise=False) -> float:
    """Physical growth rate ln|lambda| / beta of wavenumber k (T = beta t, Eq. scaling)."""
    lam = hydro_eigenvalue(Q, alpha, beta, tau, k, 0.0, dm_variant, precise)
    return math.log(abs(lam)) / beta


def t_plus_one(tau: float) -> dict:
    """T_i + 1 for i = 1..6 from the defining series."""
    return {i: t_series(i, tau) + 1.0 for i in range(1, 7)}


def predicted_error_coefficients(Q: int, alpha: float, beta: float, tau: float) -> tuple[float, float]:
    """(E4, E6): the truncation error predicted by Sec. 2.2, written as
    E4 d^4 rho/dX^4 + E6 d^6 rho/dX^6 on the right-hand side of the KS equation
    (advection ignored, as there).
    D1Q5: Eq. KS_trunc11 + Eq. KS_trunc2.
    D1Q7: Eq. remained_truc_error_KS (delta f^eq and delta M cancel the rest)."""
    T = t_plus_one(tau)
    e6_beta0 = alpha ** 4 * T[6] / (90.0 * T[2])
    e6_beta1 = beta * (T[2] / T[1] - T[3] / T[2] - T[5] / T[4])
    if Q == 5:
        e4 = beta * (T[2] / (2.0 * T[1]) - T[3] / T[2])
        e6 = e6_beta0 - alpha ** 2 * T[6] / (6.0 * T[4]) + e6_beta1
    else:
        e4 = 0.0
        e6 = e6_beta0 + e6_beta1
    return e4, e6


def max_growth(Q, alpha, beta, tau, rho_bars=(0.0,), nk=256, dm_variant=lbks.DM_DERIVED) -> float:
    """Largest physical growth rate ln(max |lambda|)/beta over all Q branches,
    kappa in (0, pi] and the given background states."""
    best = -np.inf
    kap = np.linspace(np.pi / nk, np.pi, nk)
    for rb in rho_bars:
        a = linearised_a(Q, alpha, beta, tau, rb, dm_variant)
        for kp in kap:
            lam = np.linalg.eigvals(amplification_matrix(Q, a, tau, kp))
            best = max(best, float(np.max(np.log(np.abs(lam)))) / beta)
    return best


def linearly_stable(Q, alpha, beta, tau, rho_bars=(0.0,), slack=1.05, nk=256, dm_variant=lbks.DM_DERIVED) -> bool:
    """Reading of "stable" used here: no linear mode grows faster than `slack`
    times the KS maximum growth rate 1/4 (reached at k = 1/sqrt 2)."""
    return max_growth(Q, alpha, beta, tau, rho_bars, nk, dm_variant) <= slack * 0.25


def critical_dt(Q, alpha, tau, lo=1e-9, hi=1e-1, rho_bars=(0.0,), iters=40) -> float:
    """Largest beta (by bisection in log beta) that is linearly stable; assumes
    stability is monotone in beta on [lo, hi]."""
    if not linearly_stable(Q, alpha, lo, tau, rho_bars):
        return 0.0
    a, b = math.log(lo), math.log(hi)
    for _ in range(iters):
        m = 0.5 * (a + b)
        if linearly_stable(Q, alpha, math.exp(m), tau, rho_bars):
            a = m
        else:
            b = m
    return math.exp(a)


def linear_evolution(Q, alpha, beta, tau, kappa, nsteps, dm_variant=lbks.DM_DERIVED) -> complex:
    """1^T G(kappa)^n A: the factor multiplying exp(i kappa x) in rho after n
    steps from f = f^eq(eps exp(i kappa x)) / eps, with J = 0."""
    A, _ = lbks.feq_linear_quadratic(Q, alpha, beta, tau, dm_variant, advection=False)
    G = amplification_matrix(Q, A, tau, kappa)
    v = A.astype(np.complex128)
    Gn = np.linalg.matrix_power(G, int(nsteps))
    return complex(np.sum(Gn @ v))


def tau_fit(Q: int, dX: float, dT: float) -> float:
    """Minimum stable tau fitted in Sec. 3, Eq. general_tau_formula with
    Eq. A_B_fit_D1Q5 / Eq. A_B_fit_D1Q7."""
    if Q == 5:
        A, B = 0.103 * dX ** -0.381, -13.2 * dX + 6.56
    else:
        A, B = 0.0886 * dX ** -0.472, -12.5 * dX + 6.64
    lg = math.log10(dT)
    return A * (lg + B) ** 2 + 1.0 if lg >= -B else 1.0


def tau_fit_critical_dt(Q: int, dX: float) -> float:
    """End of the tau = 1 branch of the fit: 10^(-B)."""
    B = -13.2 * dX + 6.56 if Q == 5 else -12.5 * dX + 6.64
    return 10.0 ** (-B)
