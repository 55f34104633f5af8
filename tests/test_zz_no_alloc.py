"""The allocation-free mass/energy entry point (lb_ks_mass_energy_noalloc)
gives the same FP64 mass and energy as lb_ks_mass_energy on the same state.

That entry point exists for callers that cannot allocate device memory (an
application that owns all device memory through its own pool, a monitoring
hook that must work when the device is out of memory): its scratch is a
static device array shared by all calls.  This file is collected last so a
failure here leaves every other test already run; it passes both alone in a
fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

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


def _f16_scale(lb, Q, r0, dx, dt, tau):
    """The run's FP16 storage scale: the largest |g_i| of the initial state f = f^eq(rho0),
    g_0 taken against the initial mean (the storage offset)."""
    A, B, _ = lb.lb_ks_params(Q, dx, dt, tau)
    rb = float(np.mean(r0))
    g = [A[i] * r0 + B[i] * r0 * r0 - (rb if i == 0 else 0.0) for i in range(Q)]
    return max(float(np.abs(gi).max()) for gi in g)


@pytest.mark.parametrize("prec,elem", [(0, np.float64), (1, np.float32), (2, np.float16)])
def test_noalloc_matches_handle_reduction(lb, prec, elem):
    N, Q = 5003, 7
    rng = np.random.default_rng(21)
    r0 = 0.3 + 0.05 * rng.standard_normal(N)
    h = lb.lb_ks_init(Q, N, N * 0.1, 1e-4, 1.7, r0, lb.lb_ks_default_opts(precision=prec, recentre_every=0))
    try:
        lb.lb_ks_step(h, 300)
        ref = np.empty(1), np.empty(1)
        lb.lb_ks_mass_energy(h, ref[0], ref[1])
        buf = np.zeros(lb.lb_ks_state_bytes(h), dtype=np.uint8)
        lb.lb_ks_save(h, buf)
    finally:
        lb.lb_ks_free(h)
    # populations section of the checkpoint: Q planes of plane = N rounded up to 32 elements
    plane = (N + 31) // 32 * 32
    nbytes = Q * plane * np.dtype(elem).itemsize
    pops = buf[-nbytes:].view(elem)
    f = torch.from_numpy(pops.copy()).cuda()
    rhobar = 0.0 if prec == 0 else sum(r0.tolist()) / N  # the run's initial mean (storage offset)
    scale = _f16_scale(lb, Q, r0, 0.1, 1e-4, 1.7) if prec == 2 else 1.0
    # FP16: the handle sums the scaled halves in float-float pairs, this entry point in
    # FP64; both take every term as the same float product, so they agree to the pairs'
    # ~2^-48 (the scale derived here may differ from the run's in its last bits)
    rel = 1e-12 if prec != 2 else 1e-9
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out.zero_()
        lb.lb_ks_mass_energy_noalloc(Q, prec, f, plane, N, rhobar, scale, out)
        m, e = out.cpu().numpy()
        assert m == pytest.approx(ref[0][0], rel=rel, abs=1e-12)
        assert e == pytest.approx(ref[1][0], rel=rel)
    host = np.zeros(2)
    lb.lb_ks_mass_energy_noalloc(Q, prec, f, plane, N, rhobar, scale, host)
    np.testing.assert_array_equal(host, out.cpu().numpy())
    if prec != 2:  # only FP16 storage is scaled
        with pytest.raises(lb.LbKsError) as e:
            lb.lb_ks_mass_energy_noalloc(Q, prec, f, plane, N, rhobar, 2.0, host)
        assert e.value.code == -1


@pytest.mark.parametrize("prec,elem", [(1, np.float32), (2, np.float16)])
def test_noalloc_at_its_largest_size(lb, prec, elem):
    """N = 2^24 exactly: every one of the 16384 tile slots of the static scratch is
    used.  The populations are seeded values; the reference is the FP64 sum of the
    same stored values (each scaled by the same float product for FP16)."""
    N, Q = 1 << 24, 7
    plane = N + 64
    rng = np.random.default_rng(33)
    pops = (0.05 * rng.standard_normal((Q, plane))).astype(elem)
    scale = 0.75 if prec == 2 else 1.0
    rhobar = 0.125
    vals = pops[:, :N].astype(np.float32) * np.float32(scale)  # the float product each term takes
    rho = rhobar + vals.astype(np.float64).sum(axis=0)
    f = torch.from_numpy(pops.reshape(-1)).cuda()
    out = np.zeros(2)
    for _ in range(2):
        lb.lb_ks_mass_energy_noalloc(Q, prec, f, plane, N, rhobar, scale, out)
        assert out[0] == pytest.approx(rho.sum(), rel=1e-12)
        assert out[1] == pytest.approx(np.dot(rho, rho), rel=1e-12)


def test_noalloc_rejects_sizes_beyond_its_scratch(lb):
    f = torch.zeros(7 * 64, dtype=torch.float64, device="cuda")
    out = np.zeros(2)
    with pytest.raises(lb.LbKsError) as e:
        lb.lb_ks_mass_energy_noalloc(7, 0, f, (1 << 24) + 1, (1 << 24) + 1, 0.0, 1.0, out)
    assert e.value.code == -1
