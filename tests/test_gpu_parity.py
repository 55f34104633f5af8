"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances:
 * FP64 (all kernel families): max |rho_GPU - rho_oracle| <= 1e-12 after 1000
   steps of the 512-site two-harmonic workload (the bar the method's FP64
   implementation is held to); elsewhere 1e-12 relative to max |rho|.
 * The three kernel families run the same fused arithmetic, so with equal
   storage precision they agree bitwise.
 * FP32: the collision conserves mass exactly in the rounded arithmetic, so
   what is left is unbiased rounding: each step rounds Q populations by
   <= 2^-24 relative, a random walk over n steps.  The tests bound rel-L2 by
   sqrt(n Q) 2^-24 exp(T/4), exp(T/4) being the largest linear amplification
   of KS over T = n dt.
"""
import numpy as np
import pytest

from oracle import lbks as ora

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L32 = 32 * np.pi


@pytest.fixture(scope="module")
def lb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03540_gb300 import build

    build.build()
    import paper_1711_03540_gb300 as lb

    return lb


def run_gpu(lb, Q, N, L, dt, tau, rho0, n, **opts):
    N = np.atleast_1d(np.asarray(N, dtype=np.int64))
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), N.shape).copy()
    dt = np.broadcast_to(np.asarray(dt, dtype=np.float64), N.shape).copy()
    tau = np.broadcast_to(np.asarray(tau, dtype=np.float64), N.shape).copy()
    h = lb.lb_ks_batch_init(Q, N, L, dt, tau, np.ascontiguousarray(rho0, dtype=np.float64), lb.lb_ks_default_opts(**opts))
    try:
        lb.lb_ks_step(h, n)
        out = np.empty(int(N.sum()))
        lb.lb_ks_rho(h, out)
        desc = lb.lb_ks_describe(h)
    finally:
        lb.lb_ks_free(h)
    return out, desc


def two_harmonic(N, L=L32):
    X = np.arange(N) * (L / N)
    return np.cos(X / 16) * (1 + np.sin(X / 16))


KERNELS = {"plain": 1, "stream": 2, "resident": 3}


@pytest.mark.parametrize("kern", ["plain", "stream", "resident"])
def test_fp64_512_sites_1000_steps_matches_oracle(lb, kern):
    N, dt, tau = 512, 5e-5, 1.0
    r0 = two_harmonic(N)
    ref = ora.run(5, r0, L32 / N, dt, tau, 1000)
    out, desc = run_gpu(lb, 5, N, L32, dt, tau, r0, 1000, kernel=KERNELS[kern])
    assert desc["kernel"] == KERNELS[kern]
    assert np.max(np.abs(out - ref)) <= 1e-12
    assert abs(out.sum() - r0.sum()) <= 1e-12 * np.abs(r0).sum()


@pytest.mark.parametrize("Q", [5, 7])
@pytest.mark.parametrize("kern,S,NT", [("plain", 0, 0), ("stream", 0, 0), ("resident", 8, 256), ("resident", 4, 64),
                                       ("resident", 6, 96)])
def test_fp64_ragged_batch_matches_oracle(lb, Q, kern, S, NT):
    """Uneven lattice lengths (primes, the minimum 2 c_max + 1, tile edges, and
    lengths that force the resident kernel to split lattices into segments)."""
    cm = (Q - 1) // 2
    Ns = np.array([2 * cm + 1, 13, 97, 255, 256, 257, 1023, 1025, 2049, 3001], dtype=np.int64)
    rng = np.random.default_rng(11)
    r0 = np.concatenate([0.3 * rng.standard_normal(n) + 0.1 for n in Ns])
    dx = np.linspace(0.3, 0.6, Ns.size)
    Ls = Ns * dx
    dts = np.full(Ns.size, 2e-4)
    taus = np.linspace(1.0, 2.0, Ns.size)
    n = 300
    ref, _ = ora.run_batch(Q, Ns, dx, dts, taus, r0, n)
    out, desc = run_gpu(lb, Q, Ns, Ls, dts, taus, r0, n, kernel=KERNELS[kern], sites_per_thread=S,
                        threads_per_block=NT, steps_per_launch=37 if kern == "resident" else 0)
    assert desc["kernel"] == KERNELS[kern]
    assert np.max(np.abs(out - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("prec", [0, 1])
def test_kernel_families_agree_bitwise(lb, prec):
    Ns = np.array([300, 777, 1500, 5000], dtype=np.int64)
    rng = np.random.default_rng(3)
    r0 = np.concatenate([0.01 * rng.standard_normal(n) for n in Ns])
    args = (7, Ns, Ns * 0.1, np.full(4, 1e-4), np.array([1.5, 2.0, 2.5, 3.0]), r0, 200)
    outs = [run_gpu(lb, *args, precision=prec, kernel=k)[0] for k in (1, 2, 3)]
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    seg = run_gpu(lb, *args, precision=prec, kernel=3, threads_per_block=64, steps_per_launch=16)[0]
    np.testing.assert_array_equal(outs[0], seg)


@pytest.mark.parametrize("n", [240, 228])
def test_two_lane_resident_schedule_bitwise(lb, n):
    """Whole lattices and segmented ones run as two concurrent lanes (rings: one
    launch per chunk, in place when the segment lane makes an even number of
    launches; segments: many short launches).  Both parities of the segment
    launch count give the plain kernel's result bitwise."""
    Ns = np.array([300, 700, 3000, 5000], dtype=np.int64)
    rng = np.random.default_rng(31)
    r0 = np.concatenate([0.01 * rng.standard_normal(k) for k in Ns])
    args = (7, Ns, Ns * 0.1, np.full(4, 1e-4), np.array([1.5, 2.0, 2.5, 3.0]), r0, n)
    ref = run_gpu(lb, *args, precision=1, kernel=1)[0]
    out, desc = run_gpu(lb, *args, precision=1, kernel=3, threads_per_block=64)
    assert desc["kernel"] == 3
    np.testing.assert_array_equal(ref, out)


def test_autotuned_handle_starts_from_rho0(lb):
    """The autotuner times its trials on the not yet initialised arenas; the run
    that follows must start from f^eq(rho0) with zero steps done, and every tiling
    computes the same arithmetic, so the result equals the plain kernel's bitwise."""
    Ns = np.array([300, 2000, 5000, 7000], dtype=np.int64)
    rng = np.random.default_rng(41)
    r0 = np.concatenate([0.01 * rng.standard_normal(k) for k in Ns])
    args = (7, Ns, Ns * 0.1, np.full(4, 1e-4), np.array([1.5, 2.0, 2.5, 3.0]), r0, 300)
    ref = run_gpu(lb, *args, precision=1, kernel=1, recentre_every=100)[0]
    out, desc = run_gpu(lb, *args, precision=1, kernel=3, recentre_every=100, autotune=1)
    assert desc["kernel"] == 3
    np.testing.assert_array_equal(ref, out)


@pytest.mark.parametrize("Q", [5, 7])
def test_f16s_resident_one_step_per_launch_equals_stream(lb, Q):
    """Scaled FP16: the streaming step (FP16 tile, two sites per store) equals the
    resident kernel at one step per launch bitwise, on even and odd tile tails."""
    Ns = np.array([640, 2000, 1027, 333, Q, 4097, 2048], dtype=np.int64)
    rng = np.random.default_rng(4)
    r0 = np.concatenate([0.01 * rng.standard_normal(n) for n in Ns])
    args = (Q, Ns, Ns * 0.1, np.full(Ns.size, 1e-4), np.linspace(1.5, 2.5, Ns.size), r0, 50)
    a = run_gpu(lb, *args, precision=2, kernel=2)[0]
    b = run_gpu(lb, *args, precision=2, kernel=3, steps_per_launch=1)[0]
    np.testing.assert_array_equal(a, b)


def test_f16s_stream_many_tiles_per_block_equals_resident(lb):
    """Scaled FP16 on 1.18 M sites in 1158 streaming tiles of 1024 sites (ragged tails,
    lattices from 7 to 2^18 sites, the resident kernel holding the long ones as
    segments): the streaming step equals the resident kernel at one step per launch
    bitwise."""
    rng = np.random.default_rng(44)
    Ns = np.array([1 << 18, 7, 262147, 5000, 1 << 17, 99999, 333, 2048 * 97 + 5, 1 << 16, 4097, 7, 150001],
                  dtype=np.int64)
    r0 = np.concatenate([0.01 * rng.standard_normal(n) for n in Ns])
    tiles = int(sum((n + 1023) // 1024 for n in Ns))
    assert tiles == 1158
    args = (7, Ns, Ns * 0.1, np.full(Ns.size, 1e-4), np.linspace(1.5, 2.5, Ns.size), r0, 20)
    a, da = run_gpu(lb, *args, precision=2, kernel=2)
    b = run_gpu(lb, *args, precision=2, kernel=3, steps_per_launch=1)[0]
    assert da["kernel"] == 2
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("kern", [2, 3])
def test_fp32_error_against_oracle(lb, kern):
    Ns = np.array([256, 1000, 4000, 8192], dtype=np.int64)
    from paper_1711_03540_gb300 import workloads

    rng = np.random.default_rng(5)
    r0 = np.concatenate([workloads.random_modes(int(n), n * 0.1, rng) for n in Ns])
    taus = np.array([1.5, 2.0, 2.5, 3.0])
    n, dt = 2000, 1e-4
    ref, _ = ora.run_batch(7, Ns, np.full(4, 0.1), np.full(4, dt), taus, r0, n)
    out, _ = run_gpu(lb, 7, Ns, Ns * 0.1, dt, taus, r0, n, precision=1, kernel=kern, recentre_every=500)
    off = np.concatenate([[0], np.cumsum(Ns)])
    bound = np.sqrt(n * 7) * 2.0 ** -24 * np.exp(n * dt / 4)
    for i in range(Ns.size):
        a, b = out[off[i]:off[i + 1]], ref[off[i]:off[i + 1]]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= bound


@pytest.mark.parametrize("kern,kpl", [(3, 500), (3, 100), (2, 1)])
def test_f16s_error_against_oracle(lb, kern, kpl):
    """Scaled FP16 storage (FP32 arithmetic; populations stored as g / scale in FP16,
    scale per lattice) against the FP64 oracle on the lattices of the FP32 test.  The
    state is rounded to FP16 E times: once at initialisation, then at every launch
    edge of the resident kernel (kpl steps per launch) or after every step of the
    streaming kernel; each rounding moves a stored value by at most half an ulp,
    2^-12 of it, so the error is bounded by a random walk of E Q roundings of ulp
    2^-11, amplified at most by the largest KS growth rate 1/4:
    sqrt(E Q) 2^-11 exp(T/4).  (The FP32 arithmetic adds sqrt(n Q) 2^-24.)"""
    Ns = np.array([256, 1000, 4000, 8192], dtype=np.int64)
    from paper_1711_03540_gb300 import workloads

    rng = np.random.default_rng(5)
    r0 = np.concatenate([workloads.random_modes(int(n), n * 0.1, rng) for n in Ns])
    taus = np.array([1.5, 2.0, 2.5, 3.0])
    n, dt = 2000, 1e-4
    ref, _ = ora.run_batch(7, Ns, np.full(4, 0.1), np.full(4, dt), taus, r0, n)
    out, _ = run_gpu(lb, 7, Ns, Ns * 0.1, dt, taus, r0, n, precision=2, kernel=kern, recentre_every=500,
                     steps_per_launch=kpl if kern == 3 else 0)
    off = np.concatenate([[0], np.cumsum(Ns)])
    E = 1 + (n // kpl)
    bound = np.sqrt(E * 7) * 2.0 ** -11 * np.exp(n * dt / 4) + np.sqrt(n * 7) * 2.0 ** -24
    for i in range(Ns.size):
        a, b = out[off[i]:off[i + 1]], ref[off[i]:off[i + 1]]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= bound, (Ns[i], bound)


def test_printed_delta_m_variant_matches_oracle_and_differs(lb):
    """The printed reading of Eq. delta_M is kept as an option: the GPU follows the
    oracle with the same reading, and the two readings differ once tau != 1."""
    N, L, dt, tau, n = 400, 40.0, 1e-4, 2.0, 500
    r0 = two_harmonic(N, L)
    ref_p = ora.run(7, r0, L / N, dt, tau, n, dm_variant=ora.DM_PRINTED)
    ref_d = ora.run(7, r0, L / N, dt, tau, n)
    out_p, _ = run_gpu(lb, 7, N, L, dt, tau, r0, n, dm_variant=1, kernel=3)
    assert np.max(np.abs(out_p - ref_p)) <= 1e-12 * np.abs(ref_p).max()
    assert np.max(np.abs(ref_p - ref_d)) > 1e-9 * np.abs(ref_d).max()


def test_full_inverse_weight_ablation_matches_oracle(lb):
    """The weight ablation (full 7-speed inverse for D1Q7's w1, w2, w4) runs on the
    GPU with the oracle's same reading; it differs from the default reading."""
    N, L, dt, tau, n = 400, 40.0, 1e-4, 2.0, 500
    r0 = two_harmonic(N, L)
    ref_f = ora.run(7, r0, L / N, dt, tau, n, dm_variant=ora.WEIGHTS_FULL_INVERSE)
    ref_d = ora.run(7, r0, L / N, dt, tau, n)
    for kern in (1, 3):
        out, _ = run_gpu(lb, 7, N, L, dt, tau, r0, n, dm_variant=lb.WEIGHTS_FULL_INVERSE, kernel=kern)
        assert np.max(np.abs(out - ref_f)) <= 1e-12 * np.abs(ref_f).max()
    assert np.max(np.abs(ref_f - ref_d)) > 1e-9 * np.abs(ref_d).max()


def test_zero_steps_returns_initial_density(lb):
    r0 = two_harmonic(100)
    for prec in (0, 1):
        out, _ = run_gpu(lb, 7, 100, 10.0, 1e-4, 1.5, r0, 0, precision=prec)
        assert np.max(np.abs(out - r0)) <= (1e-14 if prec == 0 else 1e-6)


def test_split_calls_equal_one_call_and_graph_replay(lb):
    Ns = np.array([500, 3000], dtype=np.int64)
    rng = np.random.default_rng(8)
    r0 = np.concatenate([0.01 * rng.standard_normal(n) for n in Ns])
    base = dict(precision=1, recentre_every=64)
    for kern in (2, 3):
        h1 = lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(2, 1e-4), np.array([2.0, 2.5]), r0,
                                 lb.lb_ks_default_opts(kernel=kern, **base))
        h2 = lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(2, 1e-4), np.array([2.0, 2.5]), r0,
                                 lb.lb_ks_default_opts(kernel=kern, use_graph=0, **base))
        try:
            for _ in range(5):
                lb.lb_ks_step(h1, 100)  # graphs replayed after the first capture
            for _ in range(10):
                lb.lb_ks_step(h2, 50)
            a, b = np.empty(r0.size), np.empty(r0.size)
            lb.lb_ks_rho(h1, a)
            lb.lb_ks_rho(h2, b)
            assert lb.lb_ks_steps_done(h1) == lb.lb_ks_steps_done(h2) == 500
        finally:
            lb.lb_ks_free(h1)
            lb.lb_ks_free(h2)
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_checkpoint_resume_bitwise(lb, prec):
    Ns = np.array([700, 2500], dtype=np.int64)
    rng = np.random.default_rng(9)
    r0 = np.concatenate([0.01 * rng.standard_normal(n) for n in Ns])
    mk = lambda: lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(2, 1e-4), np.array([1.7, 2.9]), r0,
                                     lb.lb_ks_default_opts(precision=prec, recentre_every=100 if prec else 0))
    a, b = mk(), mk()
    try:
        lb.lb_ks_step(a, 1000)
        lb.lb_ks_step(b, 500)
        buf = np.zeros(lb.lb_ks_state_bytes(b), dtype=np.uint8)
        lb.lb_ks_save(b, buf)
        lb.lb_ks_free(b)
        b = mk()
        lb.lb_ks_load(b, buf)
        assert lb.lb_ks_steps_done(b) == 500
        lb.lb_ks_step(b, 500)
        ra, rb = np.empty(r0.size), np.empty(r0.size)
        lb.lb_ks_rho(a, ra)
        lb.lb_ks_rho(b, rb)
    finally:
        lb.lb_ks_free(a)
        lb.lb_ks_free(b)
    np.testing.assert_array_equal(ra, rb)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_checkpoint_load_validates_and_rebases_guard_phase(lb, use_graph):
    """A checkpoint taken 400 steps after a guard of a handle that recentres every 500
    loads into one that recentres every 100 (phase 400 mod 100 = 0: guards 100 and 200
    steps on, after which the mass is the initial one to the storage granularity) and
    steps on; a record that moves a run in the arenas, a non-finite constant or a
    negative step counter gives EINVAL and leaves the handle as it was."""
    Ns = np.array([700, 2500], dtype=np.int64)
    rng = np.random.default_rng(5)
    r0 = np.concatenate([0.01 * rng.standard_normal(n) for n in Ns])
    mk = lambda every: lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(2, 1e-4), np.array([1.7, 2.9]), r0,
                                           lb.lb_ks_default_opts(precision=1, recentre_every=every,
                                                                 use_graph=use_graph))
    a = mk(500)
    b = None
    try:
        lb.lb_ks_step(a, 400)
        buf = np.zeros(lb.lb_ks_state_bytes(a), dtype=np.uint8)
        lb.lb_ks_save(a, buf)
        b = mk(100)
        plane = int(sum((n + 31) // 32 * 32 for n in Ns))
        rec = (buf.size - 64 - 16 * Ns.size - 4 * 7 * plane) // Ns.size  # bytes of one run record
        base = 64 + 8 * Ns.size  # the run records: off (int64) first, N, then a[0] (double)
        for corrupt, why in (
                (lambda v: v[base + rec:base + rec + 8].view(np.int64).__iadd__(32), "layout differs"),
                (lambda v: v[base + 16:base + 24].view(np.float64).__setitem__(0, np.nan), "not finite"),
                (lambda v: v[40:48].view(np.int64).__setitem__(0, -1), "negative")):
            bad = buf.copy()
            corrupt(bad)
            with pytest.raises(lb.LbKsError) as e:
                lb.lb_ks_load(b, bad)
            assert e.value.code == -1 and why in lb.lb_ks_last_error(b)
            assert lb.lb_ks_steps_done(b) == 0
        lb.lb_ks_load(b, buf)
        assert lb.lb_ks_steps_done(b) == 400
        lb.lb_ks_step(b, 200)
        mb = np.empty(2)
        lb.lb_ks_mass_energy(b, mb, None)  # right after the guard 200 steps on
        lb.lb_ks_step(b, 50)
        assert lb.lb_ks_steps_done(b) == 650
        rb = np.empty(r0.size)
        lb.lb_ks_rho(b, rb)
    finally:
        lb.lb_ks_free(a)
        if b is not None:
            lb.lb_ks_free(b)
    assert np.all(np.isfinite(rb))
    m0 = np.array([r0[:700].sum(), r0[700:].sum()])
    assert np.all(np.abs(mb - m0) <= 2 * np.ceil(Ns / 1024) * 2.0 ** -24)


def _mass_after(lb, Ns, r0, prec, every, n):
    # streaming kernel: the populations are rounded to the storage precision every step
    h = lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(Ns.size, 1e-4), np.linspace(1.5, 3.0, Ns.size), r0,
                            lb.lb_ks_default_opts(precision=prec, recentre_every=every, kernel=2))
    try:
        lb.lb_ks_step(h, n)
        m, e = np.empty(Ns.size), np.empty(Ns.size)
        lb.lb_ks_mass_energy(h, m, e)
    finally:
        lb.lb_ks_free(h)
    assert np.all(e > 0)
    return m


def test_recentring_holds_the_mass(lb):
    """The FP64 guard returns every run's mass to its initial value (the
    invariant sum_i f^eq_i = rho) at each guard step, to within the storage
    granularity: rounding residuals are carried along each 1024-site tile, so at
    most one half-ulp of g_0 per tile remains."""
    Ns = np.array([1000, 3000, 6000], dtype=np.int64)
    rng = np.random.default_rng(12)
    r0 = np.concatenate([0.5 + 0.01 * rng.standard_normal(n) for n in Ns])
    off = np.concatenate([[0], np.cumsum(Ns)])
    m0 = np.array([r0[off[i]:off[i + 1]].sum() for i in range(Ns.size)])
    for prec, ulp in ((1, 2.0 ** -24), (2, 2.0 ** -11)):
        guarded = np.abs(_mass_after(lb, Ns, r0, prec, 250, 2000) - m0)
        assert np.all(guarded <= 2 * np.ceil(Ns / 1024) * ulp * 1.0)  # |g_0| < 1 here
        if prec == 2:  # FP16 storage drifts visibly without the guard
            free = np.abs(_mass_after(lb, Ns, r0, prec, 0, 2000) - m0)
            assert np.all(free > 10 * guarded)


def test_device_pointers_and_torch_stream(lb):
    N = 2048
    r0 = torch.tensor(two_harmonic(N, 204.8), dtype=torch.float64, device="cuda")
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    h = lb.lb_ks_init(7, N, 204.8, 1e-4, 1.5, r0, lb.lb_ks_default_opts(stream=s))
    try:
        lb.lb_ks_step(h, 200)
        lb.lb_ks_rho(h, out)
    finally:
        lb.lb_ks_free(h)
    ref = ora.run(7, r0.cpu().numpy(), 0.1, 1e-4, 1.5, 200)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12 * np.abs(ref).max()


def test_unstable_run_is_reported_and_sticky(lb):
    """A time step far beyond the stability limit blows up; the FP64 guard sees a
    non-finite mass, and the handle then reports LB_KS_EUNSTABLE on every call."""
    N = 256
    r0 = 0.5 * np.cos(2 * np.pi * 7 * np.arange(N) / N)
    h = lb.lb_ks_init(5, N, N * 0.05, 5e-2, 1.0, r0, lb.lb_ks_default_opts(precision=1, recentre_every=50))
    try:
        lb.lb_ks_step(h, 5000)
        with pytest.raises(lb.LbKsError) as e:
            lb.lb_ks_rho(h, np.empty(N))
        assert e.value.code == -4
        with pytest.raises(lb.LbKsError) as e:
            lb.lb_ks_step(h, 1)
        assert e.value.code == -4
    finally:
        lb.lb_ks_free(h)


def test_init_warns_about_linearly_unstable_runs(lb):
    """The handle is created either way; last_error starts with "warning:" when the
    linear check flags a run (D1Q7, dx = 0.1, dt = 1e-4 needs tau above ~1.5)."""
    r0 = two_harmonic(64, 6.4)
    h = lb.lb_ks_init(7, 64, 6.4, 1e-4, 1.0, r0)
    try:
        assert lb.lb_ks_last_error(h).startswith("warning:")
    finally:
        lb.lb_ks_free(h)
    h = lb.lb_ks_init(7, 64, 6.4, 1e-4, 1.6, r0)
    try:
        assert lb.lb_ks_last_error(h) == "no error"
    finally:
        lb.lb_ks_free(h)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_nonfinite_rho0_is_einval_naming_the_first_run(lb, prec):
    """rho0's finiteness is checked on the device (with its mass, mean and FP16 scale):
    a NaN in run 2 and an Inf in run 3 give EINVAL naming run 2, and no handle."""
    Ns = np.array([64, 100, 80, 90], dtype=np.int64)
    r0 = 0.01 * np.random.default_rng(9).standard_normal(int(Ns.sum()))
    r0[64 + 100 + 5] = np.nan
    r0[64 + 100 + 80 + 3] = np.inf
    with pytest.raises(lb.LbKsError) as e:
        lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(4, 1e-4), np.full(4, 2.0), r0,
                            lb.lb_ks_default_opts(precision=prec, kernel=lb.KERNEL_RESIDENT))
    assert e.value.code == -1
    assert "run 2: rho0 is not finite" in lb.lb_ks_last_error(None)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_rho_into_pinned_device_and_pageable_memory_agree(lb, precision):
    """lb_ks_rho gathers into device memory directly, into pinned host memory in chunks of
    tiles copied out while the next chunk is gathered, and into other host memory through
    one staged copy: the three give the same values bitwise, on a batch whose chunk
    boundaries fall inside runs."""
    Ns = np.array([5000, 37, 1 << 15, 12345, 777, 40000, 7, 3001], dtype=np.int64)
    rng = np.random.default_rng(46)
    r0 = np.concatenate([0.01 * rng.standard_normal(n) for n in Ns])
    h = lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(Ns.size, 1e-4), np.linspace(1.5, 2.5, Ns.size),
                            r0, lb.lb_ks_default_opts(precision=precision, kernel=2))
    try:
        lb.lb_ks_step(h, 30)
        pageable = np.empty(int(Ns.sum()))
        lb.lb_ks_rho(h, pageable)
        pinned = torch.full((int(Ns.sum()),), np.nan, dtype=torch.float64).pin_memory()
        lb.lb_ks_rho(h, pinned)
        dev = torch.full((int(Ns.sum()),), np.nan, dtype=torch.float64, device="cuda")
        lb.lb_ks_rho(h, dev)
    finally:
        lb.lb_ks_free(h)
    assert np.all(np.isfinite(pageable))
    np.testing.assert_array_equal(pinned.numpy(), pageable)
    np.testing.assert_array_equal(dev.cpu().numpy(), pageable)
