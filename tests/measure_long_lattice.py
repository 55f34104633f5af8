"""Measurement for the single large lattice: D1Q7, N = 2^24 sites, Delta X = 0.1,
Delta T = 1e-4, tau = 1.51, 64 random modes with k <= 1.2 (workloads.long_lattice).
Relative L2 error of FP32 and scaled-FP16 storage (streaming and register-resident
kernels, FP64 guard every 500 steps) against FP64 at T = 1, 2, 5, 10; the FP64
reference is the GPU's plain FP64 kernel (parity-tested against the oracle to
1e-12; the oracle itself would need hours for 1.7e12 site-updates).

    python tests/measure_long_lattice.py [--t-end 10]

prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def snapshots(lb, wl, times, **opts):
    h = lb.lb_ks_batch_init(wl.scheme, wl.N, wl.L, wl.dt, wl.tau, wl.rho0, lb.lb_ks_default_opts(**opts))
    out, done, sec = {}, 0, 0.0
    rho = np.empty(int(wl.N.sum()))
    try:
        for T in times:
            n = int(round(T / wl.dt[0]))
            t0 = time.perf_counter()
            lb.lb_ks_step(h, n - done)
            lb.lb_ks_rho(h, rho)
            sec += time.perf_counter() - t0
            done = n
            out[T] = rho.copy()
        desc = lb.lb_ks_describe(h)
    finally:
        lb.lb_ks_free(h)
    return out, sec, desc


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--t-end", type=float, default=10.0)
    args = p.parse_args()
    from paper_1711_03540_gb300 import build, workloads

    build.build()
    import paper_1711_03540_gb300 as lb

    wl = workloads.long_lattice()
    times = [t for t in (1, 2, 5, 10) if t <= args.t_end]
    ref, sec64, _ = snapshots(lb, wl, times, precision=lb.F64, kernel=lb.KERNEL_PLAIN)
    res = {"workload": wl.name, "sites": int(wl.N.sum()), "T": times,
           "fp64_plain": {"seconds": sec64}}
    for name, opts in (("fp32_resident", dict(precision=lb.F32, kernel=lb.KERNEL_RESIDENT)),
                       ("fp32_stream", dict(precision=lb.F32, kernel=lb.KERNEL_STREAM)),
                       ("f16s_resident", dict(precision=lb.F16S, kernel=lb.KERNEL_RESIDENT)),
                       ("f16s_stream", dict(precision=lb.F16S, kernel=lb.KERNEL_STREAM))):
        got, sec, desc = snapshots(lb, wl, times, recentre_every=500, **opts)
        res[name] = {"seconds": sec, "kernel": desc["kernel"],
                     "rel_l2": {str(T): float(np.linalg.norm(got[T] - ref[T]) / np.linalg.norm(ref[T])) for T in times}}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
