"""Each plausible mistake, planted in the oracle (on the CPU), is caught by
at least one of the pins above.  Guards against pins that a broken oracle
would still pass."""
import numpy as np
import pytest

from oracle import analysis, front, lbks


def _front_G(Q, alpha=0.4, beta=2e-5, T=1.0):
    X = front.nodes(alpha)
    r = lbks.run(Q, front.rho_exact(X, 0.0), alpha, beta, 1.0, int(round(T / beta)), boundary="reservoir",
                 rho_left=front.RHO_LEFT, rho_right=front.RHO_RIGHT)
    return front.global_relative_error(r[1:-1], front.rho_exact(X[1:-1], T))


@pytest.mark.parametrize("m", [1, 4])
def test_front_catches_streaming_direction_and_advection_sign(m):
    good = _front_G(5)
    with lbks.mutation(m):
        bad = _front_G(5)
    assert good < 2e-3 and bad > 50 * good


def test_growth_rate_catches_dropped_k_term():
    k = 0.5
    good = analysis.growth_rate(5, 0.1, 1e-6, 1.0, k)
    with lbks.mutation(3):
        bad = analysis.growth_rate(5, 0.1, 1e-6, 1.0, k)
    exact = k * k - k ** 4
    assert abs(good - exact) < 1e-3 and abs(bad - exact) > 0.1


def test_dispersion_catches_dropped_delta_feq():
    """Without delta f^eq the D1Q7 k^6 error is D1Q5's alpha^2 term again."""
    alpha, beta, tau = 0.1, 1e-4, 1.5
    _, e6 = analysis.predicted_error_coefficients(7, alpha, beta, tau)
    k = 0.2
    exact = k * k - k ** 4
    good = analysis.growth_rate(7, alpha, beta, tau, k, precise=True) - exact
    with lbks.mutation(5):
        bad = analysis.growth_rate(7, alpha, beta, tau, k, precise=True) - exact
    assert abs(good) < 3 * abs(e6) * k ** 6
    assert abs(bad) > 20 * abs(e6) * k ** 6


def test_growth_rate_catches_dropped_m_term():
    """Without M w4 the hyperdiffusion -k^4 of KS is gone from the growth rate."""
    k = 0.5
    good = analysis.growth_rate(5, 0.1, 1e-6, 1.0, k)
    with lbks.mutation(6):
        bad = analysis.growth_rate(5, 0.1, 1e-6, 1.0, k)
    exact = k * k - k ** 4
    assert abs(good - exact) < 1e-3 and abs(bad - exact - k ** 4) < 1e-3


def test_dispersion_catches_dropped_delta_m():
    """delta M exists to cancel the beta d^4 error of Eq. KS_trunc2: without it the
    D1Q7 growth rate carries D1Q5's beta k^4 error term again."""
    alpha, beta, tau = 0.1, 1e-4, 1.5
    _, e6 = analysis.predicted_error_coefficients(7, alpha, beta, tau)
    e4_q5, _ = analysis.predicted_error_coefficients(5, alpha, beta, tau)
    k = 0.2
    exact = k * k - k ** 4
    good = analysis.growth_rate(7, alpha, beta, tau, k, precise=True) - exact
    with lbks.mutation(7):
        bad = analysis.growth_rate(7, alpha, beta, tau, k, precise=True) - exact
    assert abs(good) < 3 * abs(e6) * k ** 6
    assert abs(bad) > 8 * abs(e6) * k ** 6
    assert abs(bad - e4_q5 * k ** 4) < 0.2 * abs(e4_q5 * k ** 4)


@pytest.mark.parametrize("Q,tau", [(5, 1.7), (7, 2.5)])
def test_matrix_power_catches_relaxation_by_tau(Q, tau):
    """Relaxing by tau instead of 1/tau (the same at tau = 1, so the pin runs at
    tau != 1): the step no longer follows the amplification matrix built with 1/tau."""
    N, m, n = 64, 3, 400
    alpha, beta = 0.2, 1e-4
    kappa = 2 * np.pi * m / N
    x = np.arange(N)
    eps = 1e-2
    expect = eps * np.real(analysis.linear_evolution(Q, alpha, beta, tau, kappa, n) * np.exp(1j * kappa * x))
    good = lbks.run(Q, eps * np.cos(kappa * x), alpha, beta, tau, n, advection=False)
    with lbks.mutation(8):
        bad = lbks.run(Q, eps * np.cos(kappa * x), alpha, beta, tau, n, advection=False)
    assert np.max(np.abs(good - expect)) < 1e-13
    assert not np.all(np.abs(bad - expect) < 1e-6)


def test_front_catches_exchanged_w1_entries():
    """w1 with its c = +2 and c = -2 entries exchanged has first moment 5/3, not 1:
    the advection, and so the front's speed, is wrong."""
    good = _front_G(5)
    with lbks.mutation(9):
        bad = _front_G(5)
    assert good < 2e-3 and bad > 20 * good


@pytest.mark.parametrize("Q", [5, 7])
def test_front_catches_linear_advection(Q):
    """rho J w1 in place of rho^2 J w1 makes the advection of KS linear; the travelling
    front of Table 5 exists only through that nonlinearity."""
    good = _front_G(Q)
    with lbks.mutation(10):
        bad = _front_G(Q)
    assert good < 2e-3 and bad > 50 * good
