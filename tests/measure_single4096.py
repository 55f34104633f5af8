"""Measurement for the single-lattice D1Q7 configuration (N = 4096 on L = 32 pi,
rho0 = cos(X/16)(1 + sin(X/16)), tau = 3, Delta T = 5e-6, FP64): accuracy against a
pseudo-spectral ETDRK4 solution (1024 modes, h = 1e-3; oracle/spectral.py) as a
function of T, and the accuracy-versus-cost frontier of D1Q5 and D1Q7.

The paper compares the schemes at equal accuracy (Sec. 3, Table 6): a larger tau
allows a larger step, but the error grows with tau.  So both schemes run at
tau in {1, 1.5, 2, 2.5, 3, 4}, each at 0.8 x its linear critical time step
(oracle/analysis.critical_dt), to T = 1; for each D1Q7 point the cheapest D1Q5
point that is at least as accurate gives the cost ratio at equal accuracy.

    python tests/measure_single4096.py [--t-end 150]

prints one JSON line.  Uses the GPU (C ABI, plain FP64 kernel: one lattice) and
the oracle's spectral solver and stability analysis on the host.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import analysis  # noqa: E402
from oracle.spectral import ETDRK4  # noqa: E402

L = 32 * np.pi
N_LB, N_SPEC = 4096, 1024


def rho0(X):
    return np.cos(X / 16.0) * (1.0 + np.sin(X / 16.0))


def spectral_snapshots(times, h=1e-3):
    """ETDRK4 solution on the 1024-point grid at the given times."""
    X = np.arange(N_SPEC) * (L / N_SPEC)
    s = ETDRK4(N_SPEC, L, h)
    v = np.fft.rfft(rho0(X))
    out, t_steps = {}, 0
    for T in sorted(times):
        n = int(round(T / h))
        while t_steps < n:
            v = s.step(v)
            t_steps += 1
        out[T] = np.fft.irfft(v, n=N_SPEC)
    return out


def lb_snapshots(lb, Q, tau, dt, times):
    """GPU run; rho at the given times on the LB grid, and the seconds per unit T."""
    X = np.arange(N_LB) * (L / N_LB)
    h = lb.lb_ks_init(Q, N_LB, L, dt, tau, rho0(X), lb.lb_ks_default_opts(kernel=lb.KERNEL_PLAIN))
    out, done, sec = {}, 0, 0.0
    try:
        rho = np.empty(N_LB)
        for T in sorted(times):
            n = int(round(T / dt))
            t0 = time.perf_counter()
            lb.lb_ks_step(h, n - done)
            lb.lb_ks_rho(h, rho)  # waits for the stream
            sec += time.perf_counter() - t0
            done = n
            out[T] = rho.copy()
    finally:
        lb.lb_ks_free(h)
    return out, sec / max(times)


def rel_err(lb_rho, spec_rho):
    a = lb_rho[:: N_LB // N_SPEC]  # LB nodes that coincide with the spectral grid
    return float(np.linalg.norm(a - spec_rho) / np.linalg.norm(spec_rho))


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--t-end", type=float, default=150.0)
    args = p.parse_args()
    from paper_1711_03540_gb300 import build

    build.build()
    import paper_1711_03540_gb300 as lb

    alpha = L / N_LB
    times7 = [t for t in (1, 2, 5, 10, 20, 50, 100, 150) if t <= args.t_end]
    spec = spectral_snapshots(times7)
    s7, sec7 = lb_snapshots(lb, 7, 3.0, 5e-6, times7)
    d1q7 = {"tau": 3.0, "dt": 5e-6, "seconds_per_unit_T": sec7,
            "rel_l2_vs_etdrk4": {str(T): rel_err(s7[T], spec[T]) for T in times7}}
    # accuracy-versus-cost frontier of both schemes at T = 1: each tau at 0.8 x its
    # linear critical time step
    frontier = {5: [], 7: []}
    for Q in (5, 7):
        for tau in (1.0, 1.5, 2.0, 2.5, 3.0, 4.0):
            dt = 0.8 * analysis.critical_dt(Q, alpha, tau)
            sn, sec = lb_snapshots(lb, Q, tau, dt, [1])
            frontier[Q].append({"tau": tau, "dt": dt, "seconds_per_unit_T": sec,
                                "rel_l2_vs_etdrk4_T1": rel_err(sn[1], spec[1])})
    # for each D1Q7 point: the cheapest D1Q5 point at least as accurate
    ratios = []
    for r7 in frontier[7]:
        ok = [r5 for r5 in frontier[5] if r5["rel_l2_vs_etdrk4_T1"] <= r7["rel_l2_vs_etdrk4_T1"]]
        if ok:
            r5 = min(ok, key=lambda r: r["seconds_per_unit_T"])
            ratios.append({"d1q7_tau": r7["tau"], "d1q5_tau": r5["tau"],
                           "cost_ratio_d1q5_over_d1q7": r5["seconds_per_unit_T"] / r7["seconds_per_unit_T"]})
    print(json.dumps({"config": "d1q7_n4096_l32pi (FP64, plain kernel)", "d1q7_cfg": d1q7,
                      "frontier_d1q5": frontier[5], "frontier_d1q7": frontier[7], "equal_accuracy": ratios}))


if __name__ == "__main__":
    main()
