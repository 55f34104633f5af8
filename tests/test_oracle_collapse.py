"""Pin of the tau = 1 collapse (the state is rho alone) against the oracle's full
LB scheme.

At tau = 1 the BGK collision of Eq. LB_equation_ordinary leaves f*_i = f^eq_i(rho),
so after streaming rho'(x) = sum_i f^eq_i(rho(x - c_i)).  With f^eq_i = A_i rho +
B_i rho^2, A_i even and B_i odd in c_i (Sec. 2, the weight tables of the appendix),
and sum_i A_i = 1, sum_i B_i = 0, the +c and -c planes pair into

    rho'(x) = rho(x) + sum_{c=1}^{c_max} { A_c [rho(x-c) + rho(x+c) - 2 rho(x)]
                                          + B_c [rho(x-c) - rho(x+c)] [rho(x-c) + rho(x+c)] }.

The test restates that stencil in numpy (independent of the oracle's arithmetic)
and checks it against the oracle's LB runs at tau = 1, periodic and with the
fixed-value ends of the front test (Sec. 3).  It fails if the oracle dropped a
term of f^eq, flipped the sign of B, streamed the wrong way, or if the reading
of the reservoir ends changed.
"""
import numpy as np
import pytest

from oracle import front, lbks as ora


def stencil_step(rho, A, B, cmax, periodic=True, rho_left=0.0, rho_right=0.0):
    """One step of the collapsed scheme; reservoir mode holds nodes 0 and N-1 (and
    everything beyond) at the end values."""
    N = rho.size
    if periodic:
        ext = np.concatenate([rho[-cmax:], rho, rho[:cmax]])
    else:
        ext = np.concatenate([np.full(cmax, rho_left), rho, np.full(cmax, rho_right)])
        ext[cmax] = rho_left
        ext[cmax + N - 1] = rho_right
    mid = ext[cmax:cmax + N]
    out = mid.copy()
    for c in range(1, cmax + 1):
        lo, hi = ext[cmax - c:cmax - c + N], ext[cmax + c:cmax + c + N]
        out += A[2 * c - 1] * (lo + hi - 2 * mid) + B[2 * c - 1] * (lo - hi) * (lo + hi)
    if not periodic:
        out[0], out[-1] = rho_left, rho_right
    return out


@pytest.mark.parametrize("Q", [5, 7])
def test_coefficient_symmetries_behind_the_collapse(Q):
    A, B = ora.feq_linear_quadratic(Q, 0.2, 5e-5, 1.0)
    for c in range(1, (Q - 1) // 2 + 1):
        assert A[2 * c - 1] == A[2 * c]
        assert B[2 * c - 1] == -B[2 * c]
    assert abs(A.sum() - 1.0) < 1e-13 and abs(B.sum()) < 1e-16


@pytest.mark.parametrize("Q", [5, 7])
def test_collapse_equals_oracle_lb_at_tau_one_periodic(Q):
    rng = np.random.default_rng(17)
    N, alpha, beta, n = 200, 0.2, 5e-5, 400
    X = np.arange(N) * alpha
    rho0 = 0.5 * np.cos(2 * np.pi * 3 * X / (N * alpha)) + 0.1 * rng.standard_normal(N) + 0.3
    A, B = ora.feq_linear_quadratic(Q, alpha, beta, 1.0)
    r = rho0.copy()
    for _ in range(n):
        r = stencil_step(r, A, B, (Q - 1) // 2)
    ref = ora.run(Q, rho0, alpha, beta, 1.0, n)
    assert np.max(np.abs(r - ref)) <= 1e-12 * np.abs(ref).max()
    # mass: the paired form conserves sum rho exactly in exact arithmetic
    assert abs(r.sum() - rho0.sum()) <= 1e-11 * np.abs(rho0).sum()


@pytest.mark.parametrize("Q", [5, 7])
def test_collapse_equals_oracle_lb_at_tau_one_reservoir(Q):
    alpha, beta, n = 0.4, 2e-5, 2000
    X = front.nodes(alpha)
    rho0 = front.rho_exact(X, 0.0)
    A, B = ora.feq_linear_quadratic(Q, alpha, beta, 1.0)
    r = rho0.copy()
    for _ in range(n):
        r = stencil_step(r, A, B, (Q - 1) // 2, periodic=False, rho_left=front.RHO_LEFT, rho_right=front.RHO_RIGHT)
    ref = ora.run(Q, rho0, alpha, beta, 1.0, n, boundary="reservoir", rho_left=front.RHO_LEFT,
                  rho_right=front.RHO_RIGHT)
    assert np.max(np.abs(r - ref)) <= 1e-12 * np.abs(ref).max()


def test_collapse_differs_from_lb_away_from_tau_one():
    """The identity is special to tau = 1: at tau = 1.5 the LB state is not f^eq."""
    Q, N, alpha, beta, n = 7, 128, 0.2, 5e-5, 50
    rng = np.random.default_rng(3)
    rho0 = 0.1 * rng.standard_normal(N)
    A, B = ora.feq_linear_quadratic(Q, alpha, beta, 1.5)
    r = rho0.copy()
    for _ in range(n):
        r = stencil_step(r, A, B, 3)
    ref = ora.run(Q, rho0, alpha, beta, 1.5, n)
    assert np.max(np.abs(r - ref)) > 1e-6 * np.abs(ref).max()
