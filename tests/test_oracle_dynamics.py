"""Pins of the oracle's time step against what the mathematics fixes:
exact mass conservation, exact linear evolution (matrix power of the
amplification matrix), reflection and translation symmetry, the KS
growth rate k^2 - k^4 (Eq. KS_eq) and the truncation errors predicted in
Sec. 2.2 (Eq. KS_trunc11, Eq. KS_trunc2, Eq. delta_M, Eq.
remained_truc_error_KS), and the stability ordering of Sec. 3."""
import math

import numpy as np
import pytest

from oracle import analysis, lbks

L1 = 32 * np.pi


def rho0_cfg1(N, L=L1):
    X = np.arange(N) * (L / N)
    return np.cos(X / 16) * (1 + np.sin(X / 16))


@pytest.mark.parametrize("Q", [5, 7])
def test_mass_conserved_10k_steps(Q):
    N = 512
    alpha = L1 / N
    r0 = rho0_cfg1(N) + 0.37  # non-zero mean, so the sum is not trivially zero
    r = lbks.run(Q, r0, alpha, 5e-5, 1.0 if Q == 5 else 1.3, 10000)
    scale = np.sum(np.abs(r0))
    assert abs(np.sum(r) - np.sum(r0)) <= 1e-12 * scale
    assert np.all(np.isfinite(r))


@pytest.mark.parametrize("Q,tau", [(5, 1.0), (5, 1.7), (7, 1.0), (7, 2.5)])
def test_linear_evolution_matches_matrix_power(Q, tau):
    """With J = 0 the step is linear and translation invariant, so a single
    mode evolves by G(kappa)^n exactly (up to rounding)."""
    N, m, n = 64, 3, 400
    alpha, beta = 0.2, 1e-4
    kappa = 2 * np.pi * m / N
    x = np.arange(N)
    eps = 1e-2
    r = lbks.run(Q, eps * np.cos(kappa * x), alpha, beta, tau, n, advection=False)
    amp = analysis.linear_evolution(Q, alpha, beta, tau, kappa, n)
    expect = eps * np.real(amp * np.exp(1j * kappa * x))
    assert np.max(np.abs(r - expect)) < 1e-13


@pytest.mark.parametrize("Q", [5, 7])
def test_reflection_symmetry(Q):
    """KS is invariant under X -> -X, rho -> -rho; with even w0,w2,w4,w6 and odd w1
    the LB step is too: rho0(x) -> -rho0(-x) gives -rho(-x, t)."""
    N = 200
    rng = np.random.default_rng(5)
    r0 = 0.5 * rng.standard_normal(N)
    refl = lambda a: -np.roll(a[::-1], 1)  # a(x) -> -a(-x mod N)
    a = lbks.run(Q, r0, 0.3, 1e-4, 1.4, 3000)
    b = lbks.run(Q, refl(r0), 0.3, 1e-4, 1.4, 3000)
    assert np.max(np.abs(b - refl(a))) < 1e-13


def test_translation_invariance_bitwise():
    N = 150
    rng = np.random.default_rng(6)
    r0 = rng.standard_normal(N)
    a = lbks.run(7, r0, 0.3, 1e-4, 1.4, 500)
    b = lbks.run(7, np.roll(r0, 17), 0.3, 1e-4, 1.4, 500)
    np.testing.assert_array_equal(np.roll(a, 17), b)


@pytest.mark.parametrize("Q", [5, 7])
def test_growth_rate_tends_to_ks(Q):
    """ln|lambda|/beta -> k^2 - k^4 as alpha, beta -> 0 (Eq. KS_eq, Eq. taylor_result)."""
    errs = []
    for alpha in (0.2, 0.1, 0.05):
        beta = alpha ** 4 / 100
        g = [analysis.growth_rate(Q, alpha, beta, 1.0, k, precise=True) for k in (0.3, 0.7071, 1.0)]
        exact = [k * k - k ** 4 for k in (0.3, 0.7071, 1.0)]
        errs.append(max(abs(a - b) for a, b in zip(g, exact)))
    # D1Q5 converges at second order in alpha (the alpha^2 d6 term of Eq. KS_trunc11),
    # D1Q7 faster (that term is removed)
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
    assert errs[2] < (5e-4 if Q == 5 else 2e-6)


def _fit_error_coefficients(Q, alpha, beta, tau, dm_variant=lbks.DM_DERIVED):
    ks = np.array([0.05, 0.1, 0.15, 0.2])
    err = np.array([analysis.growth_rate(Q, alpha, beta, tau, k, dm_variant, precise=True) - (k * k - k ** 4)
                    for k in ks])
    coef = np.linalg.lstsq(np.stack([ks ** 4, ks ** 6, ks ** 8], 1), err, rcond=None)[0]
    return coef[0], coef[1]


CASES = [(0.1, 1e-4, 2.0), (0.2, 1e-3, 1.5), (0.1, 1e-4, 1.5)]


@pytest.mark.parametrize("alpha,beta,tau", CASES)
def test_d1q5_truncation_error_matches_taylor_prediction(alpha, beta, tau):
    """The k^4 and k^6 error coefficients of the D1Q5 growth rate are the ones
    of Eq. KS_trunc2 (beta d4) and Eq. KS_trunc11 + Eq. KS_trunc2 (d6)."""
    c4, c6 = _fit_error_coefficients(5, alpha, beta, tau)
    e4, e6 = analysis.predicted_error_coefficients(5, alpha, beta, tau)
    assert c4 == pytest.approx(e4, rel=2e-3)
    assert c6 == pytest.approx(-e6, rel=2e-3)


@pytest.mark.parametrize("alpha,beta,tau", CASES)
def test_d1q7_removes_k4_error(alpha, beta, tau):
    """delta M (Eq. delta_M, bracket read with (T2+1)) removes the beta d4 error:
    the fitted k^4 coefficient is orders of magnitude below beta; the printed
    (T4+1) bracket leaves a k^4 error of order beta (reading recorded in the
    oracle header)."""
    c4, c6 = _fit_error_coefficients(7, alpha, beta, tau)
    c4p, _ = _fit_error_coefficients(7, alpha, beta, tau, lbks.DM_PRINTED)
    assert abs(c4) < 1e-2 * beta
    assert abs(c4p) > 1.0 * beta
    # and the remaining d6 coefficient is Eq. remained_truc_error_KS to leading order
    _, e6 = analysis.predicted_error_coefficients(7, alpha, beta, tau)
    assert c6 == pytest.approx(-e6, rel=0.35)
    # D1Q7 error is far below D1Q5's at the same (alpha, beta, tau)
    c4_5, c6_5 = _fit_error_coefficients(5, alpha, beta, tau)
    assert abs(c6) < 0.1 * abs(c6_5)


def test_stability_ordering_at_dx_0p1():
    """Sec. 3: at Delta X = 0.1, tau = 1, D1Q7 tolerates a smaller Delta T than
    D1Q5, and both exceed the sufficient bound alpha^4/90 = 1.11e-6
    (Eq. cond_stability).  Checked here with the linear criterion."""
    d5 = analysis.critical_dt(5, 0.1, 1.0, lo=1e-7, hi=1e-3, iters=18)
    d7 = analysis.critical_dt(7, 0.1, 1.0, lo=1e-7, hi=1e-3, iters=18)
    assert d7 < d5
    assert d7 > 0.1 ** 4 / 90


def test_full_inverse_weights_satisfy_the_moment_rule_and_give_the_printed_w5_w6():
    """Appendix A: the full 7-speed inverse (Eq. cond_weight for p = 0..6); the paper
    prints only its w5 and w6, which the oracle's D1Q7 set uses."""
    c = lbks.speeds(7).astype(float)
    for l in range(7):
        w = lbks.weight_full(l)
        for p in range(7):
            assert abs((c ** p * w).sum() - (1.0 if p == l else 0.0)) < 1e-12
    np.testing.assert_array_equal(lbks.weight_full(5), lbks.weight(7, 5))
    np.testing.assert_array_equal(lbks.weight_full(6), lbks.weight(7, 6))


@pytest.mark.parametrize("alpha,beta,tau", CASES)
def test_full_inverse_weights_flip_the_alpha2_d6_error(alpha, beta, tau):
    """The weight reading of Sec. 2.3 (a negative control): with the D1Q5 sets padded
    with zeros at c = +-3, delta f^eq removes the alpha^2 d6 error of D1Q5; with the
    full 7-speed inverse (whose 6th moments vanish) the same delta f^eq leaves that
    error at D1Q5's size with the opposite sign."""
    _, c6_5 = _fit_error_coefficients(5, alpha, beta, tau)
    _, c6_pad = _fit_error_coefficients(7, alpha, beta, tau)
    c4_full, c6_full = _fit_error_coefficients(7, alpha, beta, tau, lbks.WEIGHTS_FULL_INVERSE)
    assert abs(c6_pad) < 0.02 * abs(c6_5)
    assert c6_full == pytest.approx(-c6_5, rel=0.05)
    assert abs(c4_full) < 1e-2 * beta  # delta M still removes the beta d4 term
