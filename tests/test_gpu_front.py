"""The travelling-front test of Sec. 3 (Table 5) on the GPU: lattices with
fixed-value ends (lb_ks_batch_init_reservoir), checked against the oracle's
reservoir mode (FP64: 1e-12 relative) and against the analytic solution
through the global relative error G of Sec. 3."""
import numpy as np
import pytest

from oracle import front, lbks as ora

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03540_gb300 import build

    build.build()
    import paper_1711_03540_gb300 as lb

    return lb


def _gpu_front(lb, Q, alphas, beta, tau, n, **opts):
    Ns = np.array([int(round(60.0 / a)) + 1 for a in alphas], dtype=np.int64)
    r0 = np.concatenate([front.rho_exact(front.nodes(a), 0.0) for a in alphas])
    k = len(alphas)
    h = lb.lb_ks_batch_init_reservoir(Q, Ns, np.full(k, 60.0), np.full(k, beta), np.full(k, tau), r0,
                                      np.full(k, front.RHO_LEFT), np.full(k, front.RHO_RIGHT),
                                      lb.lb_ks_default_opts(**opts))
    try:
        lb.lb_ks_step(h, n)
        out = np.empty(r0.size)
        lb.lb_ks_rho(h, out)
    finally:
        lb.lb_ks_free(h)
    off = np.concatenate([[0], np.cumsum(Ns)])
    return [out[off[i]:off[i + 1]] for i in range(k)]


@pytest.mark.parametrize("Q", [5, 7])
def test_front_fp64_matches_oracle_reservoir_mode(lb, Q):
    alphas, beta, tau, n = [0.4, 0.3, 0.2], 2e-5, 1.0, 5000
    got = _gpu_front(lb, Q, alphas, beta, tau, n)
    for a, g in zip(alphas, got):
        X = front.nodes(a)
        ref = ora.run(Q, front.rho_exact(X, 0.0), a, beta, tau, n, boundary="reservoir",
                      rho_left=front.RHO_LEFT, rho_right=front.RHO_RIGHT)
        assert np.max(np.abs(g - ref)) <= 1e-12 * np.abs(ref).max()
        assert g[0] == pytest.approx(front.RHO_LEFT, rel=1e-15) and g[-1] == pytest.approx(front.RHO_RIGHT, rel=1e-15)


def test_front_global_error_on_gpu(lb):
    """Sec. 3: both schemes follow the analytic front; at tau = 1 and small Delta T
    D1Q7's G is far below D1Q5's, in FP64 and in FP32 storage."""
    alphas, beta, T = [0.4, 0.2], 2e-5, 1.0
    n = int(round(T / beta))
    G = {}
    for Q in (5, 7):
        for prec in (0, 1):
            got = _gpu_front(lb, Q, alphas, beta, 1.0, n, precision=prec)
            for a, g in zip(alphas, got):
                X = front.nodes(a)
                G[(Q, prec, a)] = front.global_relative_error(g[1:-1], front.rho_exact(X[1:-1], T))
    for prec in (0, 1):
        for a in alphas:
            assert G[(7, prec, a)] < 0.2 * G[(5, prec, a)]
        assert G[(5, prec, 0.2)] < G[(5, prec, 0.4)]
    # FP32 storage adds its own rounding error (~1e-4 relative after 5e4 steps of a
    # field whose mean is 3) on top of the scheme's truncation error
    for key in [(5, 0.2), (7, 0.2), (5, 0.4), (7, 0.4)]:
        assert abs(G[(key[0], 1, key[1])] - G[(key[0], 0, key[1])]) <= 1e-4
