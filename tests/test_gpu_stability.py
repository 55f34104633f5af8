"""The stability and accuracy map of Sec. 3 on the GPU (stability.stability_map):
batched front runs over (Delta X, Delta T, tau).

* Parity: every run of a map that straddles the stability boundary is classified
  as the oracle's reservoir-mode run of the same parameters is, and G agrees to
  1e-10 relative where the run is stable.
* The paper's findings (Sec. 3, its Figs. of tau_min and G versus Delta T and Eq.
  general_tau_formula): tau_min grows with Delta T and falls with Delta X, the
  D1Q7 scheme needs at least the tau of D1Q5, tau = 1 is stable below the fitted
  Delta T_crit, the fit is followed to within 0.35 in tau, and D1Q7's G at tau_min
  is below D1Q5's.  The fit came from the authors' runs (run length unstated), so
  only its shape and approximate values are checked.
"""
import numpy as np
import pytest

from oracle import lbks as ora

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03540_gb300 import build

    build.build()
    from paper_1711_03540_gb300 import stability

    return stability


@pytest.mark.parametrize("Q", [5, 7])
def test_map_classification_matches_oracle(st, Q):
    dx, dt, T = 0.1, 1e-4, 1.0
    taus = np.round(np.arange(1.0, 2.01, 0.1), 2)
    (p,) = st.stability_map(Q, [dx], [dt], taus, T=T)
    X = st.front_nodes(dx)
    exact = st.front_profile(X, p.T)
    assert p.steps == 10000
    assert 1.0 < p.tau_min < 2.0  # the grid straddles the boundary
    for tau, ok, G in zip(taus, p.stable, p.G_all):
        ref = ora.run(Q, st.front_profile(X, 0.0), dx, dt, float(tau), p.steps, boundary="reservoir",
                      rho_left=st.END_LEFT, rho_right=st.END_RIGHT)
        assert ok == st.is_stable(ref, exact), tau
        if ok:
            assert G == pytest.approx(st.global_relative_error(ref[1:-1], exact[1:-1]), rel=1e-10)


@pytest.fixture(scope="module")
def maps(st):
    taus = np.round(np.arange(1.0, 4.0001, 0.05), 2)
    dts = [3e-6, 3e-5, 1e-4, 3e-4]
    return {Q: st.stability_map(Q, (0.05, 0.1, 0.2), dts, taus, T=1.0, max_steps=100_000) for Q in (5, 7)}


def _grid(points):
    return {(p.dx, p.dt): p for p in points}


def test_map_follows_the_papers_fit(maps):
    for Q, pts in maps.items():
        for p in pts:
            if np.isfinite(p.tau_fit) and p.tau_fit <= 3.5:
                assert np.isfinite(p.tau_min), (Q, p.dx, p.dt)
                assert abs(p.tau_min - p.tau_fit) <= 0.35, (Q, p.dx, p.dt, p.tau_min, p.tau_fit)


def test_map_ordering(maps):
    g5, g7 = _grid(maps[5]), _grid(maps[7])
    dxs = sorted({k[0] for k in g5})
    dts = sorted({k[1] for k in g5})
    for g in (g5, g7):
        for dx in dxs:  # tau_min grows with Delta T
            t = [g[(dx, dt)].tau_min for dt in dts]
            assert all(b >= a for a, b in zip(t, t[1:])), (dx, t)
        for dt in dts:  # and falls with Delta X
            t = [g[(dx, dt)].tau_min for dx in dxs]
            assert all(b <= a for a, b in zip(t, t[1:])), (dt, t)
    for key in g5:  # D1Q7 needs at least the tau of D1Q5; its G is lower
        assert g7[key].tau_min >= g5[key].tau_min, key
        assert g7[key].G < g5[key].G, key
    # tau = 1 is stable below the fitted Delta T_crit (5.75e-6 for D1Q5 and 4.07e-6 for D1Q7 at dx = 0.1)
    assert g5[(0.1, 3e-6)].tau_min == 1.0 and g7[(0.1, 3e-6)].tau_min == 1.0
    assert g5[(0.2, 3e-6)].tau_min == 1.0 and g7[(0.2, 3e-6)].tau_min == 1.0
