"""Pins of the oracle's constants against what the paper fixes exactly:
moment conditions (Appendix A, Eq. cond_weight), the printed weight tables,
the T_i series (Sec. 2, below Eq. feq) and identities between coefficients."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import analysis, lbks

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_weights():
    rows = {}
    with open(os.path.join(GOLDEN, "weights_appendix.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            rows[(tok[0], int(tok[1]))] = [float(Fraction(t)) for t in tok[2:]]
    return rows


def test_weights_match_printed_appendix():
    g = _golden_weights()
    for l in (0, 1, 2, 3, 4):
        np.testing.assert_array_equal(lbks.weight(5, l), g[("D1Q5", l)])
        # D1Q7 uses the D1Q5 sets padded with zeros at c = +-3
        np.testing.assert_array_equal(lbks.weight(7, l), g[("D1Q5", l)] + [0.0, 0.0])
    for l in (5, 6):
        np.testing.assert_array_equal(lbks.weight(7, l), g[("D1Q7", l)])


@pytest.mark.parametrize("Q,ls", [(5, (0, 1, 2, 3, 4)), (7, (5, 6))])
def test_moment_condition(Q, ls):
    """Eq. cond_weight: sum_i c_i^p w^(l)_i = delta_pl for p < Q."""
    c = lbks.speeds(Q)
    for l in ls:
        w = lbks.weight(Q, l)
        for p in range(Q):
            assert abs(np.sum(c.astype(float) ** p * w) - (1.0 if p == l else 0.0)) < 1e-14


def test_padded_weights_higher_moments():
    """On the 7-speed lattice the padded D1Q5 sets keep their D1Q5 moments up to
    p = 4 and acquire 5th/6th moments -4 (w1, w2) and 5 (w3, w4); these are the
    terms that delta f^eq (with E = -5M) and Eq. KS_trunc11 refer to."""
    c = lbks.speeds(7).astype(float)
    m = lambda l, p: float(np.sum(c ** p * lbks.weight(7, l)))
    assert m(1, 5) == pytest.approx(-4.0, abs=1e-13)
    assert m(2, 6) == pytest.approx(-4.0, abs=1e-13)
    assert m(3, 5) == pytest.approx(5.0, abs=1e-13)
    assert m(4, 6) == pytest.approx(5.0, abs=1e-13)
    for l in (0, 1, 2, 3, 4):
        for p in range(5):
            assert m(l, p) == pytest.approx(1.0 if p == l else 0.0, abs=1e-14)


@pytest.mark.parametrize("tau", [0.75, 1.0, 1.2, 1.5, 2.0, 3.0])
def test_t_closed_forms_match_series(tau):
    co = lbks.coefficients(7, 0.1, 1e-4, tau)
    for i in (1, 2, 3, 4):
        s = analysis.t_series(i, tau)
        assert co[f"T{i}"] == pytest.approx(s, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("tau", [1.0, 1.3, 2.0, 3.0])
def test_t_plus_one_factorisations(tau):
    """T_i + 1 in factored form (algebra on Eq. T_form); T4 + 1 vanishes at the
    root of 12 tau^2 - 12 tau + 1 near 0.908, so M diverges there."""
    co = lbks.coefficients(5, 0.1, 1e-4, tau)
    assert co["T1"] + 1 == pytest.approx(tau, rel=1e-14)
    assert co["T2"] + 1 == pytest.approx(tau * (2 * tau - 1), rel=1e-14)
    assert co["T3"] + 1 == pytest.approx(tau * (6 * tau * tau - 6 * tau + 1), rel=1e-13)
    assert co["T4"] + 1 == pytest.approx(tau * (2 * tau - 1) * (12 * tau * tau - 12 * tau + 1), rel=1e-13)


@pytest.mark.parametrize("alpha,beta,tau", [(0.1, 1e-4, 1.0), (0.2, 1e-3, 1.5), (0.05, 1e-6, 3.0)])
def test_coefficient_identities(alpha, beta, tau):
    co = lbks.coefficients(7, alpha, beta, tau)
    assert co["J"] == pytest.approx(beta / (2 * alpha), rel=1e-15)
    assert co["E"] == pytest.approx(-5.0 * co["M"], rel=1e-14)
    # the scaling of Eq. scaling turns Table 2 into unit KS coefficients (Eq. taylor_result):
    T1, T2, T4 = co["T1"] + 1, co["T2"] + 1, co["T4"] + 1
    assert 0.5 * co["K"] * T2 / T1 * alpha ** 2 / beta == pytest.approx(-1.0, rel=1e-14)
    assert co["M"] / 24.0 * T4 / T1 * alpha ** 4 / beta == pytest.approx(-1.0, rel=1e-14)


def test_tau_one_values():
    a, b = 0.1, 1e-5
    co = lbks.coefficients(7, a, b, 1.0)
    assert co["K"] == pytest.approx(-2 * b / a ** 2, rel=1e-14)
    assert co["M"] == pytest.approx(-24 * b / a ** 4, rel=1e-14)
    assert co["dM"] == pytest.approx(12 * b * b / a ** 4, rel=1e-14)
    pr = lbks.coefficients(7, a, b, 1.0, dm_variant=lbks.DM_PRINTED)
    assert pr["dM"] == co["dM"]  # both readings of Eq. delta_M agree at tau = 1
    assert lbks.coefficients(5, a, b, 1.0)["dM"] == 0.0


def test_equilibrium_conserves_mass():
    """sum_i f^eq_i = rho (from the zeroth moments of the weights), for any rho."""
    for Q in (5, 7):
        for rho in (-2.0, 0.3, 5.0):
            fe = lbks.feq(Q, 0.1, 1e-4, 1.7, rho)
            assert np.sum(fe) == pytest.approx(rho, rel=1e-13)


def test_tau_fit_reproduces_printed_critical_dt():
    vals = {}
    with open(os.path.join(GOLDEN, "tau_fit_critical_dt.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            s, dx, dt = line.split()
            vals[s] = (float(dx), float(dt))
    assert analysis.tau_fit_critical_dt(5, 0.1) == pytest.approx(vals["D1Q5"][1], rel=2e-3)
    assert analysis.tau_fit_critical_dt(7, 0.1) == pytest.approx(vals["D1Q7"][1], rel=2e-3)
    assert 0.1 ** 4 / 90 == pytest.approx(vals["SUFFICIENT"][1], rel=2e-3)
    assert analysis.tau_fit(7, 0.1, 1e-4) == pytest.approx(1.5076, abs=1e-3)
    assert analysis.tau_fit(5, 0.1, 1e-7) == 1.0
