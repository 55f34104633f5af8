"""CPU tests of the stability map's host logic (paper_1711_03540_gb300.stability):
its own restatement of Table 5 and of G agrees with the oracle's, and the
classification helpers behave as documented."""
import numpy as np
import pytest

from oracle import front
from paper_1711_03540_gb300 import stability as st


@pytest.mark.parametrize("dx", [0.05, 0.1, 0.2, 0.3, 0.4])
def test_front_profile_and_nodes_match_oracle(dx):
    X = st.front_nodes(dx)
    np.testing.assert_allclose(X, front.nodes(dx), rtol=0, atol=1e-12)
    for T in (0.0, 0.5, 1.0, 5.0):
        np.testing.assert_allclose(st.front_profile(X, T), front.rho_exact(X, T), rtol=1e-15, atol=1e-15)
    assert st.END_LEFT == pytest.approx(front.RHO_LEFT, rel=1e-15)
    assert st.END_RIGHT == pytest.approx(front.RHO_RIGHT, rel=1e-15)


def test_front_profile_limits_are_the_end_values():
    """Table 5: far from the front the solution tends to the boundary values."""
    assert st.front_profile(np.array([-1e3]), 0.0)[0] == pytest.approx(st.END_LEFT, abs=1e-12)
    assert st.front_profile(np.array([1e3]), 0.0)[0] == pytest.approx(st.END_RIGHT, abs=1e-12)


def test_global_relative_error_matches_oracle():
    rng = np.random.default_rng(5)
    a, b = rng.standard_normal(300) + 3, rng.standard_normal(300) + 3
    assert st.global_relative_error(a, b) == pytest.approx(front.global_relative_error(a, b), rel=1e-15)
    assert st.global_relative_error(b, b) == 0.0


def test_min_and_max_stable_tau():
    taus = [1.0, 1.1, 1.2, 1.3, 1.4]
    assert st.min_stable_tau(taus, [0, 0, 1, 1, 1]) == 1.2
    assert st.min_stable_tau(taus, [0, 1, 0, 1, 1]) == 1.3   # an isolated stable point does not count
    assert st.min_stable_tau(taus, [1, 1, 1, 0, 0]) == 1.0   # large tau may lose accuracy
    assert st.min_stable_tau(taus, [0, 0, 0, 0, 1]) == 1.4   # the last grid point stands alone
    assert np.isnan(st.min_stable_tau(taus, [0, 0, 0, 0, 0]))
    assert st.max_stable_tau(taus, [1, 1, 1, 0, 0]) == 1.2
    assert np.isnan(st.max_stable_tau(taus, [0] * 5))


def test_is_stable():
    X = st.front_nodes(0.4)
    ex = st.front_profile(X, 0.5)
    assert st.is_stable(ex, ex)
    bad = ex.copy()
    bad[10] = np.nan
    assert not st.is_stable(bad, ex)
    big = ex.copy()
    big[10] = 3.0 + 3.0 * np.max(np.abs(ex - 3.0))
    assert not st.is_stable(big, ex)


def test_equal_accuracy_picks_plateau_and_matching_step():
    def pt(Q, dt, G):
        return st.MapPoint(Q, 0.1, dt, int(1 / dt), 1.0, 1.0, 4.0, G, 1.0)
    # D1Q5: plateau 1e-4 below dt = 1e-5, growing above; D1Q7 reaches 1e-4 up to dt = 5e-5
    p5 = [pt(5, 1e-6, 1.00e-4), pt(5, 1e-5, 1.05e-4), pt(5, 1e-4, 1e-3)]
    p7 = [pt(7, 1e-6, 1e-6), pt(7, 1e-5, 2e-5), pt(7, 5e-5, 1.0e-4), pt(7, 1e-4, 3e-4)]
    (r,) = st.equal_accuracy(p5, p7)
    assert r["d1q5_dt"] == 1e-5 and r["d1q7_dt"] == 5e-5
    assert r["step_ratio"] == pytest.approx(5.0)
    assert r["cost_ratio_d1q5_over_d1q7"] == pytest.approx(5.0 * 27 / 39)
