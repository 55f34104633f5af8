"""Error of the mixed-precision ensemble at the benchmark's full horizon: the
4096-lattice D1Q7 ensemble (N log-uniform in [256, 8192], Delta X = 0.1,
Delta T = 1e-4, tau ~ U(1.5, 3)) run for 10^5 steps (T = 10) with FP32 and with
scaled FP16 storage (resident kernel, autotuned, FP64 guard every 500 steps) against
the plain FP64 kernel (parity-tested against the oracle to 1e-12), per lattice
rel-L2 at T = 1, 2, 5, 10, the lattices with the largest errors (with how much their
FP64 solution's norm changed and the absolute RMS error), and the wall time of each leg.

    python tests/measure_ensemble_error.py [--t-end 10]

prints one JSON line.  Uses the GPU through the C ABI.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def snapshots(lb, wl, steps, **opts):
    h = lb.lb_ks_batch_init(wl.scheme, wl.N, wl.L, wl.dt, wl.tau, wl.rho0, lb.lb_ks_default_opts(**opts))
    out, done, sec = {}, 0, 0.0
    rho = np.empty(wl.sites)
    try:
        for n in steps:
            t0 = time.perf_counter()
            lb.lb_ks_step(h, n - done)
            lb.lb_ks_rho(h, rho)  # waits for the stream
            sec += time.perf_counter() - t0
            done = n
            out[n] = rho.copy()
    finally:
        lb.lb_ks_free(h)
    return out, sec


def per_run_rel_l2(wl, a, b):
    off = wl.offsets()
    return np.array([np.linalg.norm(a[off[i]:off[i + 1]] - b[off[i]:off[i + 1]]) /
                     max(np.linalg.norm(b[off[i]:off[i + 1]]), 1e-300) for i in range(wl.nruns)])


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--t-end", type=float, default=10.0)
    args = p.parse_args()
    from paper_1711_03540_gb300 import build, workloads

    build.build()
    import paper_1711_03540_gb300 as lb

    wl = workloads.ensemble(4096)
    times = [t for t in (1, 2, 5, 10) if t <= args.t_end]
    steps = [int(round(t / wl.dt[0])) for t in times]
    ref, s64 = snapshots(lb, wl, steps, precision=lb.F64, kernel=lb.KERNEL_PLAIN)
    res = {"workload": wl.name, "sites": int(wl.sites), "T": times,
           "fp64_plain": {"seconds": s64, "site_updates_per_s": wl.sites * steps[-1] / s64}}
    for name, prec in (("fp32_resident", lb.F32), ("f16s_resident", lb.F16S)):
        got, sec = snapshots(lb, wl, steps, precision=prec, kernel=lb.KERNEL_RESIDENT, recentre_every=500, autotune=1)
        errs = {str(t): per_run_rel_l2(wl, got[n], ref[n]) for t, n in zip(times, steps)}
        res[name] = {"seconds": sec, "site_updates_per_s": wl.sites * steps[-1] / sec,
                     "rel_l2_max_run": {t: float(e.max()) for t, e in errs.items()},
                     "rel_l2_median_run": {t: float(np.median(e)) for t, e in errs.items()},
                     "runs_above_1e-4": {t: int((e > 1e-4).sum()) for t, e in errs.items()}}
        # the largest errors at the last time: which lattices, how their FP64 solution's
        # norm changed since T = 0, and the absolute RMS error
        last = steps[-1]
        e = errs[str(times[-1])]
        off = wl.offsets()
        worst = np.argsort(e)[::-1][:8]
        res[name]["worst_runs"] = [
            {"run": int(i), "N": int(wl.N[i]), "rel_l2": float(e[i]),
             "norm_ratio_fp64": float(np.linalg.norm(ref[last][off[i]:off[i + 1]]) /
                                      np.linalg.norm(wl.rho0[off[i]:off[i + 1]])),
             "rms_error": float(np.sqrt(np.mean((got[last][off[i]:off[i + 1]] - ref[last][off[i]:off[i + 1]]) ** 2)))}
            for i in worst]
        nr = np.array([np.linalg.norm(ref[last][off[i]:off[i + 1]]) / np.linalg.norm(wl.rho0[off[i]:off[i + 1]])
                       for i in range(wl.nruns)])
        grow = nr >= 1.0
        res[name]["rel_l2_max_run_where_fp64_norm_did_not_decay"] = float(e[grow].max()) if grow.any() else None
        res[name]["runs_where_fp64_norm_decayed"] = int((~grow).sum())
    print(json.dumps(res))


if __name__ == "__main__":
    main()
