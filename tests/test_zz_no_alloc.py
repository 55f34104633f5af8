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


@pytest.mark.parametrize("prec,elem", [(0, np.float64), (1, np.float32)])
def test_noalloc_matches_handle_reduction(lb, prec, elem):
    N, Q = 5003, 7
    rng = np.random.default_rng(21)
    r0 = 0.3 + 0.05 * rng.standard_normal(N)
    h = lb.lb_ks_init(Q, N, N * 0.1, 1e-4, 1.7, r0, lb.lb_ks_default_opts(precision=prec))
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
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out.zero_()
        lb.lb_ks_mass_energy_noalloc(Q, prec, f, plane, N, rhobar, 1.0, out)
        m, e = out.cpu().numpy()
        assert m == pytest.approx(ref[0][0], rel=1e-12, abs=1e-12)
        assert e == pytest.approx(ref[1][0], rel=1e-12)
    host = np.zeros(2)
    lb.lb_ks_mass_energy_noalloc(Q, prec, f, plane, N, rhobar, 1.0, host)
    np.testing.assert_array_equal(host, out.cpu().numpy())


def test_noalloc_rejects_sizes_beyond_its_scratch(lb):
    f = torch.zeros(7 * 64, dtype=torch.float64, device="cuda")
    out = np.zeros(2)
    with pytest.raises(lb.LbKsError) as e:
        lb.lb_ks_mass_energy_noalloc(7, 0, f, (1 << 24) + 1, (1 << 24) + 1, 0.0, 1.0, out)
    assert e.value.code == -1
