"""GPU parity of the resident kernel's two-block work groups (thread block
clusters of 2, opts.cluster_size = 2): whole lattices of up to 2 NT S sites held
across both blocks (boundary values pushed into the other block's shared memory
every step), or as two haloed halves whose halos are exchanged every 32 steps.

* FP64: the oracle within 1e-12 relative (the same bar as the other families).
* With equal storage precision every family and work-group size runs the same
  fused arithmetic per site, so one block with segments (cluster_size = 1) and
  a cluster pair agree bitwise.
"""
import numpy as np
import pytest

from oracle import lbks as ora

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


def run_gpu(lb, Q, Ns, r0, n, taus, dx=0.1, dt=1e-4, **opts):
    Ns = np.asarray(Ns, dtype=np.int64)
    h = lb.lb_ks_batch_init(Q, Ns, Ns * dx, np.full(Ns.size, dt), np.asarray(taus, dtype=np.float64),
                            np.ascontiguousarray(r0), lb.lb_ks_default_opts(**opts))
    try:
        lb.lb_ks_step(h, n)
        out = np.empty(int(Ns.sum()))
        lb.lb_ks_rho(h, out)
        desc = lb.lb_ks_describe(h)
        desc["lanes"] = lb.lb_ks_describe_lanes(h)
    finally:
        lb.lb_ks_free(h)
    return out, desc


# S = 4, NT = 64: one block holds 256 sites, a pair 512.  Lengths just above one
# block, at the pair's maximum (V = 2 NT), with S-1-site threads, small rings that
# share a pair's bundle (and cross the block edge), and one lattice too long for a
# pair (segment lane beside the cluster lane).
PAIR_NS = [257, 300, 385, 449, 511, 512, 100, 13, 50, 200, 130, 1500]


def _inputs(Ns, seed, tau_min=1.6):
    """tau_min 1.6: above the fitted minimum stable tau of Sec. 3 (1.51 for D1Q7 at
    dx = 0.1, dt = 1e-4), so that every run stays bounded."""
    rng = np.random.default_rng(seed)
    r0 = np.concatenate([0.3 * rng.standard_normal(n) + 0.1 for n in Ns])
    taus = np.linspace(tau_min, 2.5, len(Ns))
    return r0, taus


@pytest.mark.parametrize("Q", [5, 7])
def test_cluster_pairs_fp64_match_oracle(lb, Q):
    Ns = np.array(PAIR_NS, dtype=np.int64)
    r0, taus = _inputs(Ns, 71, tau_min=1.0)  # the fitted minimum is 1.0 at dx = 0.4, dt = 2e-4
    n, dx, dt = 300, 0.4, 2e-4
    ref, _ = ora.run_batch(Q, Ns, np.full(Ns.size, dx), np.full(Ns.size, dt), taus, r0, n)
    out, desc = run_gpu(lb, Q, Ns, r0, n, taus, dx=dx, dt=dt, kernel=3, sites_per_thread=4, threads_per_block=64,
                        cluster_size=2, steps_per_launch=0)
    assert desc["kernel"] == 3 and desc["cluster_size"] == 2
    assert np.max(np.abs(out - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("S,NT", [(4, 64), (8, 96), (12, 128)])
def test_cluster_pairs_equal_single_block_segments_bitwise(lb, prec, S, NT):
    if prec == 0 and S > 8:
        pytest.skip("FP64 holds at most 8 sites per thread")
    Ns = np.array([S * NT + 1, 2 * S * NT, 2 * NT * (S - 1) + 1, S * NT // 2, 37, 5 * S * NT + 3, 1000],
                  dtype=np.int64)
    r0, taus = _inputs(Ns, 72)
    common = dict(kernel=3, precision=prec, sites_per_thread=S, threads_per_block=NT)
    one, d1 = run_gpu(lb, 7, Ns, r0, 400, taus, cluster_size=1, **common)
    two, d2 = run_gpu(lb, 7, Ns, r0, 400, taus, cluster_size=2, **common)
    plain, _ = run_gpu(lb, 7, Ns, r0, 400, taus, kernel=1, precision=prec)
    assert d1["cluster_size"] == 1 and d2["cluster_size"] == 2
    np.testing.assert_array_equal(one, plain)
    np.testing.assert_array_equal(two, plain)


# S = 4, NT = 64.  Enough pair lattices that the pairs hold most of the threads (the
# library then runs every whole lattice from one queue of pair work groups), and enough
# one-block lattices to leave single-block bundles after the pairs' spare threads are
# filled: five of them (odd) in the first set, four in the second.
MERGED_NS = [[257, 300, 385, 449, 511, 512, 400, 480, 256, 253, 192, 193, 250, 240, 200, 37, 100],
             [257, 300, 385, 449, 511, 512, 400, 480, 256, 253, 193, 250, 240, 200, 37, 100]]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("which", [0, 1])
def test_single_block_bundles_merged_into_pairs_bitwise(lb, prec, which):
    """Single-block bundles go two to a pair (the second block's pieces shifted by NT
    threads, no piece across the block edge), on one queue with the pair bundles;
    results equal the one-block plan and the plain kernel bitwise."""
    S, NT = 4, 64
    Ns = np.array(MERGED_NS[which], dtype=np.int64)
    r0, taus = _inputs(Ns, 76 + which)
    common = dict(kernel=3, precision=prec, sites_per_thread=S, threads_per_block=NT)
    one, d1 = run_gpu(lb, 7, Ns, r0, 300, taus, cluster_size=1, **common)
    two, d2 = run_gpu(lb, 7, Ns, r0, 300, taus, cluster_size=2, **common)
    plain, _ = run_gpu(lb, 7, Ns, r0, 300, taus, kernel=1, precision=prec)
    assert d1["cluster_size"] == 1 and d2["cluster_size"] == 2
    assert len(d2["lanes"]) == 1 and d2["lanes"][0]["merged_single_blocks"] == 1
    assert all(ln["merged_single_blocks"] == 0 for ln in d1["lanes"])
    np.testing.assert_array_equal(one, plain)
    np.testing.assert_array_equal(two, plain)


# S = 8, NT = 256: one block holds 2048 sites.  A lattice longer than that is held as
# two halves, one per block of the pair, each with c_max * 32 halo sites per side
# (refreshed from the other block every 32 steps) when a half with its halos fits a
# block: up to 3712 sites for D1Q7 (halo 96), 3840 for D1Q5 (halo 64); longer ones run
# as one ring across both blocks.  Small lattices fill the spare threads of both blocks.
HALVES_NS = [2049, 2500, 3001, 3500, 3712, 3900, 4096, 300, 77, 1000, 13]


@pytest.mark.parametrize("Q", [5, 7])
def test_cluster_halves_fp64_match_oracle(lb, Q):
    Ns = np.array(HALVES_NS, dtype=np.int64)
    r0, taus = _inputs(Ns, 81, tau_min=1.0)
    n, dx, dt = 300, 0.4, 2e-4
    ref, _ = ora.run_batch(Q, Ns, np.full(Ns.size, dx), np.full(Ns.size, dt), taus, r0, n)
    out, desc = run_gpu(lb, Q, Ns, r0, n, taus, dx=dx, dt=dt, kernel=3, sites_per_thread=8, threads_per_block=256,
                        cluster_size=2)
    assert desc["kernel"] == 3 and desc["cluster_size"] == 2
    assert np.max(np.abs(out - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("recentre", [0, 50])
def test_cluster_halves_bitwise_with_launch_lengths(lb, recentre):
    """F32: halves equal the plain kernel bitwise, with 1000-step launches (31 exchanges
    and a final 8-step chunk) and with 50-step launches between guards (one exchange
    and an 18-step chunk), over several graph replays."""
    Ns = np.array(HALVES_NS, dtype=np.int64)
    r0, taus = _inputs(Ns, 82)
    r0 = 0.01 * r0
    halves, d = run_gpu(lb, 7, Ns, r0, 1000, taus, kernel=3, precision=1, sites_per_thread=8, threads_per_block=256,
                        cluster_size=2, recentre_every=recentre)
    plain, _ = run_gpu(lb, 7, Ns, r0, 1000, taus, kernel=1, precision=1, recentre_every=recentre)
    assert d["cluster_size"] == 2
    # 2049 .. 3712 sites as halves, 3900 and 4096 as rings across the pair
    (pl,) = [ln for ln in d["lanes"] if ln["blocks_per_group"] == 2]
    assert pl["halved_lattices"] == 5 and pl["pair_exchange_steps"] == 32
    assert pl["steps_per_launch"] == (1000 if recentre == 0 else 50)
    np.testing.assert_array_equal(halves, plain)


def test_cluster_halves_f16s_one_step_per_launch_equals_stream(lb):
    """Scaled FP16 storage rounds at every launch edge; with one step per launch the
    halves (segments with halos, loaded and stored every step) round where the
    streaming kernel does."""
    Ns = np.array([2500, 3001, 300], dtype=np.int64)
    r0, taus = _inputs(Ns, 84)
    r0 = 0.01 * r0
    a, _ = run_gpu(lb, 7, Ns, r0, 40, taus, kernel=2, precision=2)
    b, d = run_gpu(lb, 7, Ns, r0, 40, taus, kernel=3, precision=2, sites_per_thread=8, threads_per_block=256,
                   cluster_size=2, steps_per_launch=1)
    assert sum(ln["halved_lattices"] for ln in d["lanes"]) == 2
    np.testing.assert_array_equal(a, b)


def test_cluster_halves_checkpoint(lb):
    """A checkpoint taken between launches of a run with halves restores it bitwise."""
    Ns = np.array(HALVES_NS[:7], dtype=np.int64)
    r0, taus = _inputs(Ns, 83)
    r0 = 0.01 * r0
    opts = dict(kernel=3, precision=1, sites_per_thread=8, threads_per_block=256, cluster_size=2, recentre_every=100)
    ref, _ = run_gpu(lb, 7, Ns, r0, 400, taus, **opts)
    h = lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(Ns.size, 1e-4), taus, r0, lb.lb_ks_default_opts(**opts))
    try:
        lb.lb_ks_step(h, 200)
        blob = np.empty(lb.lb_ks_state_bytes(h), dtype=np.uint8)
        lb.lb_ks_save(h, blob)
        lb.lb_ks_step(h, 200)
        a = np.empty(r0.size)
        lb.lb_ks_rho(h, a)
        lb.lb_ks_load(h, blob)
        lb.lb_ks_step(h, 200)
        b = np.empty(r0.size)
        lb.lb_ks_rho(h, b)
    finally:
        lb.lb_ks_free(h)
    np.testing.assert_array_equal(a, ref)
    np.testing.assert_array_equal(b, ref)


def test_cluster_f16s_one_step_per_launch_equals_stream(lb):
    """F16S rounds to storage at every launch edge; with one step per launch the
    pair work groups round where the streaming kernel does."""
    Ns = np.array([257, 512, 300, 60], dtype=np.int64)
    r0, taus = _inputs(Ns, 73)
    r0 = 0.01 * r0
    a, _ = run_gpu(lb, 7, Ns, r0, 40, taus, kernel=2, precision=2)
    b, d = run_gpu(lb, 7, Ns, r0, 40, taus, kernel=3, precision=2, sites_per_thread=4, threads_per_block=64,
                   cluster_size=2, steps_per_launch=1)
    assert d["cluster_size"] == 2
    np.testing.assert_array_equal(a, b)


def test_cluster_default_chooses_pairs_only_when_needed(lb):
    Ns = np.array([300, 700], dtype=np.int64)
    r0, taus = _inputs(Ns, 74)
    _, d = run_gpu(lb, 7, Ns, r0, 10, taus, kernel=3, precision=1, sites_per_thread=4, threads_per_block=64)
    assert d["cluster_size"] == 2  # 300 sites > 64 x 4
    _, d = run_gpu(lb, 7, Ns[:1] - 100, r0[:200], 10, taus[:1], kernel=3, precision=1, sites_per_thread=4,
                   threads_per_block=64)
    assert d["cluster_size"] == 1


def test_cluster_checkpoint_and_graph_replay(lb):
    """Split calls (graph replays of the pair launches, guard in between) give the
    one-call result bitwise, and a checkpoint taken midway restores it."""
    Ns = np.array([257, 512, 450, 90], dtype=np.int64)
    r0, taus = _inputs(Ns, 75)
    r0 = 0.01 * r0
    opts = dict(kernel=3, precision=1, sites_per_thread=4, threads_per_block=64, cluster_size=2, recentre_every=64)
    ref, _ = run_gpu(lb, 7, Ns, r0, 500, taus, use_graph=0, **opts)
    h = lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(4, 1e-4), taus, r0, lb.lb_ks_default_opts(**opts))
    try:
        for _ in range(3):
            lb.lb_ks_step(h, 100)
        blob = np.empty(lb.lb_ks_state_bytes(h), dtype=np.uint8)
        lb.lb_ks_save(h, blob)
        lb.lb_ks_step(h, 200)
        a = np.empty(r0.size)
        lb.lb_ks_rho(h, a)
        lb.lb_ks_load(h, blob)
        lb.lb_ks_step(h, 200)
        b = np.empty(r0.size)
        lb.lb_ks_rho(h, b)
    finally:
        lb.lb_ks_free(h)
    np.testing.assert_array_equal(a, ref)
    np.testing.assert_array_equal(b, ref)



def test_link_wait_that_runs_out_is_reported_and_the_device_stays_usable(lb):
    """Failure detection of the link between the two blocks of a pair: a lattice of 400
    sites at 4 sites x 64 threads runs as one ring across both blocks (halves with
    their 96-site halos would not fit a block).  With the testing aid, block 1 sends
    nothing across the edge at step 5 of each launch and a wait gives up after 4096
    rounds, so block 0's wait for that step runs out: the launch completes, the next
    call that checks the status reports LB_KS_ETIMEOUT, it sticks, the handle frees,
    and a new handle on the same device computes the ring bitwise as before."""
    Ns = np.array([400], dtype=np.int64)
    r0, taus = _inputs(Ns, 91)
    opts = dict(precision=1, kernel=3, sites_per_thread=4, threads_per_block=64, cluster_size=2)
    ref, desc = run_gpu(lb, 7, Ns, r0, 40, taus, **opts)
    assert desc["cluster_size"] == 2 and sum(ln["halved_lattices"] for ln in desc["lanes"]) == 0
    h = lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(1, 1e-4), taus, r0, lb.lb_ks_default_opts(**opts))
    try:
        lb.lb_ks_set_link_test(h, 5, 4096)
        lb.lb_ks_step(h, 40)
        out = np.empty(400)
        with pytest.raises(lb.LbKsError) as e:
            lb.lb_ks_rho(h, out)
        assert e.value.code == -5
        with pytest.raises(lb.LbKsError) as e:
            lb.lb_ks_step(h, 1)
        assert e.value.code == -5
    finally:
        lb.lb_ks_free(h)
    # the aid is refused once a handle has stepped
    h = lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(1, 1e-4), taus, r0, lb.lb_ks_default_opts(**opts))
    try:
        lb.lb_ks_step(h, 1)
        with pytest.raises(lb.LbKsError) as e:
            lb.lb_ks_set_link_test(h, 5, 4096)
        assert e.value.code == -1
    finally:
        lb.lb_ks_free(h)
    again, _ = run_gpu(lb, 7, Ns, r0, 40, taus, **opts)
    np.testing.assert_array_equal(again, ref)
