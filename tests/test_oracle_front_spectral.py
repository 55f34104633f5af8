"""Pins of the oracle against the analytic travelling front of Table 5 and
against an independent pseudo-spectral KS solver (ETDRK4)."""
import numpy as np
import pytest

from oracle import front, lbks, spectral


def test_front_is_an_exact_ks_solution():
    """Substitute the Table 5 solution into Eq. KS_eq symbolically."""
    sp = pytest.importorskip("sympy")
    X, T = sp.symbols("X T", real=True)
    b, X0 = 3, 20
    k = sp.Rational(1, 2) * sp.sqrt(sp.Rational(11, 19))
    th = sp.tanh(k * (X - b * T - X0))
    rho = b + sp.Rational(15, 19) * sp.sqrt(sp.Rational(11, 19)) * (-9 * th + 11 * th ** 3)
    res = sp.diff(rho, T) + rho * sp.diff(rho, X) + sp.diff(rho, X, 2) + sp.diff(rho, X, 4)
    for xv, tv in [(13.7, 0.4), (20.0, 0.0), (31.2, 2.5)]:
        assert abs(float(res.subs({X: xv, T: tv}).evalf(30))) < 1e-20
    # and the numerical transcription used by the tests agrees with it
    for xv, tv in [(13.7, 0.4), (31.2, 2.5)]:
        assert front.rho_exact(xv, tv) == pytest.approx(float(rho.subs({X: xv, T: tv})), rel=1e-14)


def test_front_boundary_values_are_its_limits():
    assert front.rho_exact(-1e3, 0.0) == pytest.approx(front.RHO_LEFT, rel=1e-14)
    assert front.rho_exact(1e3, 0.0) == pytest.approx(front.RHO_RIGHT, rel=1e-14)
    # the profile at the domain ends differs from the limits by far less than any G measured here
    assert abs(front.rho_exact(0.0, 0.0) - front.RHO_LEFT) < 1e-5


def _front_G(Q, alpha, beta, T, tau=1.0):
    X = front.nodes(alpha)
    n = int(round(T / beta))
    r = lbks.run(Q, front.rho_exact(X, 0.0), alpha, beta, tau, n, boundary="reservoir",
                 rho_left=front.RHO_LEFT, rho_right=front.RHO_RIGHT)
    return front.global_relative_error(r[1:-1], front.rho_exact(X[1:-1], T))


def test_front_global_error_small_and_converging():
    """Sec. 3: both schemes follow the analytic front; G falls as Delta X falls,
    and at tau = 1 and small Delta T the D1Q7 error is below D1Q5's (its
    alpha^2 truncation term is removed)."""
    g = {(Q, a): _front_G(Q, a, 2e-5, 1.0) for Q in (5, 7) for a in (0.4, 0.2)}
    for Q in (5, 7):
        assert g[(Q, 0.2)] < g[(Q, 0.4)]
    for a in (0.4, 0.2):
        assert g[(7, a)] < 0.2 * g[(5, a)]
    assert g[(5, 0.2)] < 1e-3 and g[(7, 0.2)] < 5e-5


def test_etdrk4_linear_mode_exact():
    L, n = 32 * np.pi, 64
    X = np.arange(n) * L / n
    k = 2 * np.pi * 7 / L
    u0 = 1e-13 * np.cos(k * X)  # small enough that the quadratic term is below rounding
    u = spectral.ETDRK4(n, L, 0.05).run(u0, 2.0)
    expect = u0 * np.exp((k * k - k ** 4) * 2.0)
    assert np.max(np.abs(u - expect)) < 1e-10 * np.max(np.abs(expect))


def test_etdrk4_fourth_order_in_time():
    L, n = 22.0, 64
    X = np.arange(n) * L / n
    u0 = np.cos(2 * np.pi * X / L) + 0.3 * np.sin(4 * np.pi * X / L)
    ref = spectral.ETDRK4(n, L, 0.0025).run(u0, 2.0)
    e1 = np.max(np.abs(spectral.ETDRK4(n, L, 0.04).run(u0, 2.0) - ref))
    e2 = np.max(np.abs(spectral.ETDRK4(n, L, 0.02).run(u0, 2.0) - ref))
    assert 10.0 < e1 / e2 < 24.0  # ~16 for a fourth-order method


def test_lb_converges_to_spectral_solution():
    """On a small periodic box (L = 32 pi, the 512-site workload's initial
    field) the LB oracle approaches the ETDRK4 solution as alpha -> 0 with
    beta ~ alpha^4 (Eq. cond_stability scaling)."""
    L, T = 32 * np.pi, 2.0
    u0 = lambda X: np.cos(X / 16) * (1 + np.sin(X / 16))
    _, at = spectral.solve(u0, L, T, n=256, h=1e-3)
    for Q in (5, 7):
        errs = []
        for N in (96, 128, 192):
            alpha = L / N
            n = int(np.ceil(T / (alpha ** 4 / 200)))
            X = np.arange(N) * alpha
            r = lbks.run(Q, u0(X), alpha, T / n, 1.0, n)
            errs.append(np.max(np.abs(r - at(X))) / np.max(np.abs(at(X))))
        assert errs[0] > errs[1] > errs[2]
        order = np.log(errs[0] / errs[2]) / np.log(192 / 96)
        assert order > 3.0
        assert errs[2] < 2e-5
