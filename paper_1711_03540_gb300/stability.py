"""Stability and accuracy map of Sec. 3: for each lattice spacing Delta X and time
step Delta T, the smallest relaxation time tau for which the travelling-front test
(Table 5) stays stable, and the global relative error G at that tau.

For each Delta T the front is run at every (Delta X, tau) pair at once, one lattice
per pair in a single batched handle with fixed-value ends
(lb_ks_batch_init_reservoir), advanced on the GPU and read back once.  A run is
called stable when every node is finite and its largest deviation from b stays
within `blowup` times that of the analytic front (unstable runs grow grid-scale
oscillations without bound).  tau_min is the smallest tau of the grid whose run
and the next grid point's run are stable (the paper records the minimum tau
required for stability); tau_max, the largest stable tau, shows where growing tau
costs accuracy (the higher-order truncation terms grow like tau^4, Sec. 2.2).

The paper records tau_min over a range of Delta T for Delta X = 0.05, 0.1, 0.2
(its Figs. for those spacings) and fits Eq. general_tau_formula; lb_ks_tau_fit
gives that fit for comparison.  The run length is not stated there; here each
Delta T runs to time T or max_steps steps, whichever comes first.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Table 5: b = 3, X_m = 0, X_M = 60, X_0 = (X_M - X_m) / 3, k = sqrt(11/19) / 2.
SPEED_B = 3.0
X_MIN, X_MAX = 0.0, 60.0
X_START = (X_MAX - X_MIN) / 3.0
WAVENUMBER = 0.5 * np.sqrt(11.0 / 19.0)
AMPLITUDE = 15.0 / 19.0 * np.sqrt(11.0 / 19.0)
END_LEFT = SPEED_B - 30.0 / 19.0 * np.sqrt(11.0 / 19.0)  # rho(X_m, t)
END_RIGHT = 2.0 * SPEED_B - END_LEFT                       # rho(X_M, t)


def front_profile(X, T: float) -> np.ndarray:
    """Table 5's analytic solution: b + A (-9 tanh z + 11 tanh^3 z), z = k (X - b T - X_0)."""
    z = np.tanh(WAVENUMBER * (np.asarray(X, dtype=np.float64) - SPEED_B * T - X_START))
    return SPEED_B + AMPLITUDE * (-9.0 * z + 11.0 * z ** 3)


def front_nodes(dx: float) -> np.ndarray:
    """Nodes X_j = X_m + j dx on [X_m, X_M], both ends included."""
    n = int(round((X_MAX - X_MIN) / dx)) + 1
    return X_MIN + np.arange(n) * ((X_MAX - X_MIN) / (n - 1))


def global_relative_error(rho_num, rho_exact) -> float:
    """Sec. 3: G = sum_x |rho^N - rho^A| / sum_x |rho^A|."""
    rho_num = np.asarray(rho_num, dtype=np.float64)
    rho_exact = np.asarray(rho_exact, dtype=np.float64)
    return float(np.abs(rho_num - rho_exact).sum() / np.abs(rho_exact).sum())


def is_stable(rho, exact, blowup: float = 2.0) -> bool:
    rho = np.asarray(rho, dtype=np.float64)
    if not np.all(np.isfinite(rho)):
        return False
    return float(np.max(np.abs(rho - SPEED_B))) <= blowup * float(np.max(np.abs(exact - SPEED_B)))


def min_stable_tau(taus, stable) -> float:
    """Smallest tau of the (ascending) grid that is stable together with the next
    grid point (or is the last one); NaN if there is none."""
    taus = np.asarray(taus, dtype=np.float64)
    stable = np.asarray(stable, dtype=bool)
    for i in range(taus.size):
        if stable[i] and (i + 1 == taus.size or stable[i + 1]):
            return float(taus[i])
    return float("nan")


def max_stable_tau(taus, stable) -> float:
    """Largest stable tau of the grid; NaN if there is none."""
    taus = np.asarray(taus, dtype=np.float64)
    stable = np.asarray(stable, dtype=bool)
    return float(taus[stable].max()) if stable.any() else float("nan")


@dataclass
class MapPoint:
    scheme: int
    dx: float
    dt: float
    steps: int
    T: float
    tau_min: float            # NaN when no tau of the grid is stable
    tau_max: float            # largest stable tau of the grid (NaN if none)
    G: float                  # global relative error at tau_min (NaN if none)
    tau_fit: float            # Eq. general_tau_formula with the paper's fitted A, B
    taus: list = field(default_factory=list)
    stable: list = field(default_factory=list)
    G_all: list = field(default_factory=list)


def stability_map(scheme: int, dxs, dts, taus, T: float = 1.0, max_steps: int = 200_000, precision: int = 0,
                  blowup: float = 2.0) -> list[MapPoint]:
    """Run the front test for every (dx, dt, tau) and return one MapPoint per (dx, dt).
    taus must be ascending and >= 1 (the library's range)."""
    from . import (lb_ks_batch_init_reservoir, lb_ks_default_opts, lb_ks_free, lb_ks_rho, lb_ks_step,
                   lb_ks_tau_fit)

    dxs = [float(v) for v in dxs]
    taus = [float(v) for v in taus]
    if any(b <= a for a, b in zip(taus, taus[1:])):
        raise ValueError("taus must be strictly ascending")
    out = []
    for dt in (float(v) for v in dts):
        n = int(max(1, min(round(T / dt), max_steps)))
        t_end = n * dt
        pairs = [(dx, tau) for dx in dxs for tau in taus]
        nodes = {dx: front_nodes(dx) for dx in dxs}
        Ns = np.array([nodes[dx].size for dx, _ in pairs], dtype=np.int64)
        rho0 = np.concatenate([front_profile(nodes[dx], 0.0) for dx, _ in pairs])
        k = len(pairs)
        h = lb_ks_batch_init_reservoir(scheme, Ns, np.full(k, X_MAX - X_MIN), np.full(k, dt),
                                       np.array([tau for _, tau in pairs]), rho0, np.full(k, END_LEFT),
                                       np.full(k, END_RIGHT), lb_ks_default_opts(precision=precision))
        try:
            lb_ks_step(h, n)
            rho = np.empty(int(Ns.sum()))
            lb_ks_rho(h, rho)
        finally:
            lb_ks_free(h)
        off = np.concatenate([[0], np.cumsum(Ns)])
        for a, dx in enumerate(dxs):
            exact = front_profile(nodes[dx], t_end)
            st, gs = [], []
            for b in range(len(taus)):
                i = a * len(taus) + b
                r = rho[off[i]:off[i + 1]]
                ok = is_stable(r, exact, blowup)
                st.append(ok)
                gs.append(global_relative_error(r[1:-1], exact[1:-1]) if ok else float("nan"))
            tmin = min_stable_tau(taus, st)
            G = gs[taus.index(tmin)] if np.isfinite(tmin) else float("nan")
            out.append(MapPoint(scheme, dx, dt, n, t_end, tmin, max_stable_tau(taus, st), G,
                                lb_ks_tau_fit(scheme, dx, dt), list(taus), st, gs))
    return out


def equal_accuracy(points5, points7, plateau_slack: float = 1.1, flop_ratio: float = 39.0 / 27.0) -> list[dict]:
    """Sec. 3's cost comparison at equal accuracy (its Table 6) from two maps of the
    same spacings, both run to the same T.  Per Delta X: D1Q5's plateau error is the
    smallest G over its Delta T grid; D1Q5 runs at the largest Delta T whose G is
    within plateau_slack of it; D1Q7 runs at the largest Delta T whose G is at most
    that D1Q5 error.  The cost ratio counts steps per unit time times the per-step
    work (flop_ratio: 39 flop per site-update for D1Q7 against 27 for D1Q5)."""
    out = []
    for dx in sorted({p.dx for p in points5}):
        p5 = [p for p in points5 if p.dx == dx and np.isfinite(p.G)]
        p7 = [p for p in points7 if p.dx == dx and np.isfinite(p.G)]
        if not p5 or not p7:
            continue
        g_plateau = min(p.G for p in p5)
        a = max((p for p in p5 if p.G <= plateau_slack * g_plateau), key=lambda p: p.dt)
        ok7 = [p for p in p7 if p.G <= a.G]
        if not ok7:
            out.append({"dx": dx, "d1q5_dt": a.dt, "d1q5_tau": a.tau_min, "G": a.G, "d1q7_dt": None})
            continue
        b = max(ok7, key=lambda p: p.dt)
        out.append({"dx": dx, "G_d1q5": a.G, "d1q5_dt": a.dt, "d1q5_tau": a.tau_min, "G_d1q7": b.G, "d1q7_dt": b.dt,
                    "d1q7_tau": b.tau_min, "step_ratio": b.dt / a.dt,
                    "cost_ratio_d1q5_over_d1q7": (b.dt / a.dt) / flop_ratio})
    return out


def main() -> None:
    """Run both schemes' maps to T = 1 on the paper's spacings and print the maps and
    the equal-accuracy comparison as one JSON line."""
    import argparse
    import json
    import time

    from . import build

    p = argparse.ArgumentParser(description="stability and accuracy map of the front test (Sec. 3)")
    p.add_argument("--T", type=float, default=1.0)
    args = p.parse_args()
    build.build()
    taus = np.round(np.arange(1.0, 4.0001, 0.05), 2)
    dts = [1e-6, 2e-6, 5e-6, 1e-5, 2e-5, 5e-5, 1e-4, 2e-4, 5e-4, 1e-3]
    dxs = (0.05, 0.1, 0.2)
    maps, secs = {}, {}
    for Q in (5, 7):
        t0 = time.perf_counter()
        maps[Q] = stability_map(Q, dxs, dts, taus, T=args.T, max_steps=10 ** 9)
        secs[Q] = time.perf_counter() - t0
    rows = [{"Q": Q, "dx": m.dx, "dt": m.dt, "steps": m.steps, "tau_min": m.tau_min, "tau_max": m.tau_max,
             "tau_fit": m.tau_fit, "G": m.G} for Q in (5, 7) for m in maps[Q]]
    print(json.dumps({"T": args.T, "seconds": secs, "map": rows, "equal_accuracy": equal_accuracy(maps[5], maps[7])}))


if __name__ == "__main__":
    main()
