"""Host logic of the multi-rank benchmark path, as world-size-2 gloo jobs on CPU.

With N GPUs each rank advances its own ensemble (the lattices are
independent, so the path shards with no collective on the data): ranks must
draw disjoint runs, the job time is the slowest rank's, and the rate counts
every rank's updates.  A rank that disappears must surface as an error on the
others (here: a barrier with a short process-group timeout), not as a hang.
"""
import datetime
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, ws, port, timeout_s=60):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=datetime.timedelta(seconds=timeout_s))


def _timing_worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    from paper_1711_03540_gb300 import workloads

    _init(rank, ws, port)
    try:
        wl = workloads.ensemble(nruns=8, nmin=256, nmax=512, seed=bench.rank_seed(workloads.BASE_SEED, rank, 8))
        my_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        t = bench.max_over_ranks(my_ms, ws, device="cpu")
        total = bench.sum_over_ranks(wl.sites * 1000, ws, device="cpu")
        rate = bench.whole_job_rate(total, t)
        out.put((rank, t, rate, wl.rho0[:16].tolist(), wl.sites))
    finally:
        dist.destroy_process_group()


def test_two_ranks_disjoint_runs_and_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_timing_worker, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    res = sorted([q.get(timeout=60) for _ in range(2)])
    (r0, t0, rate0, rho_a, sites0), (r1, t1, rate1, rho_b, sites1) = res
    assert t0 == t1 == 150.0  # both ranks report the slowest rank's time
    assert rate0 == rate1 == pytest.approx((sites0 + sites1) * 1000 / 0.150)
    assert not np.allclose(rho_a, rho_b)  # different runs on different ranks


def _dropout_worker(rank, ws, port, out):
    _init(rank, ws, port, timeout_s=5)
    if rank == 1:
        out.put((rank, "left"))
        out.close()
        out.join_thread()  # the message is flushed before the abrupt exit
        os._exit(0)  # leaves between steps, without joining the barrier
    try:
        dist.barrier()
        out.put((rank, "no error"))
    except Exception as exc:  # the survivor learns of it on the host
        out.put((rank, "error: " + type(exc).__name__))


def test_rank_dropout_surfaces_as_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dropout_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=90)
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got[1] == "left"
    assert got[0].startswith("error")
