"""Throughput of the register-resident kernel's work groups on uniform lattices and on
the benchmark ensemble (D1Q7, FP32, Delta X = 0.1, Delta T = 1e-4, tau = 2, guard every
500 steps): lattices held by one block, by a cluster pair as one ring across both
blocks, or as two haloed halves.  Each case runs 1000 steps once to warm up and capture
the graphs, then three more times; the best is printed.

    python tests/measure_work_groups.py [case ...]

cases: single4096 (152 x 8 lattices of 4096 sites, one block each), pairs8192 (608 of
8192: too long for halves with 16 sites x 256 threads, one ring across the pair),
pairs7000 and pairs5000 (608 of 7000 / 5000: two halves), ensemble (bench.py's
4096-lattice ensemble, library default plan), ensemble16 (the same at 16 x 256).
Prints one JSON line per case.  Uses the GPU through the C ABI.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

K = 152 * 8
CASES = {
    "single4096": ([4096] * K, dict(sites_per_thread=16, threads_per_block=256, cluster_size=1)),
    "pairs8192": ([8192] * (K // 2), dict(sites_per_thread=16, threads_per_block=256, cluster_size=2)),
    "pairs7000": ([7000] * (K // 2), dict(sites_per_thread=16, threads_per_block=256, cluster_size=2)),
    "pairs5000": ([5000] * (K // 2), dict(sites_per_thread=16, threads_per_block=256, cluster_size=2)),
    "ensemble": (None, dict()),
    "ensemble16": (None, dict(sites_per_thread=16, threads_per_block=256, cluster_size=2)),
}


def run(lb, torch, Ns, steps=1000, **opts):
    Ns = np.asarray(Ns, dtype=np.int64)
    r0 = 1e-2 * np.random.default_rng(1).standard_normal(int(Ns.sum()))
    o = lb.lb_ks_default_opts(precision=lb.F32, kernel=lb.KERNEL_RESIDENT, recentre_every=500, **opts)
    h = lb.lb_ks_batch_init(7, Ns, Ns * 0.1, np.full(Ns.size, 1e-4), np.full(Ns.size, 2.0), r0, o)
    try:
        lb.lb_ks_step(h, steps)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(3):
            t0 = time.perf_counter()
            lb.lb_ks_step(h, steps)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        desc, lanes = lb.lb_ks_describe(h), lb.lb_ks_describe_lanes(h)
    finally:
        lb.lb_ks_free(h)
    return float(Ns.sum()) * steps / best, desc, lanes


def main():
    import torch

    from paper_1711_03540_gb300 import build, workloads

    build.build()
    import paper_1711_03540_gb300 as lb

    for case in sys.argv[1:] or list(CASES):
        Ns, opts = CASES[case]
        if Ns is None:
            Ns = workloads.ensemble(4096).N
        v, desc, lanes = run(lb, torch, Ns, **opts)
        print(json.dumps({"case": case, "site_updates_per_s": v, "sites_per_thread": desc["sites_per_thread"],
                          "threads_per_block": desc["threads_per_block"], "lanes": lanes}), flush=True)


if __name__ == "__main__":
    main()
