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
