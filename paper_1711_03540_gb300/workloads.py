"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Shapes and distributions follow the workloads the paper's method is run on:
a single periodic lattice with a smooth two-harmonic field (the L = 32 pi
box), ensembles of uneven lattices with random low Fourier modes, and one
very long lattice whose modes lie in the band the KS equation amplifies
(k <= 1.2).  Every random draw uses numpy's PCG64 with seed
``BASE_SEED + run index``, so the tests, the benchmark and the oracle see
identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

BASE_SEED = 20171109


@dataclass
class Workload:
    name: str
    scheme: int
    N: np.ndarray     # int64 [nruns]
    L: np.ndarray     # float64 [nruns]
    dt: np.ndarray    # float64 [nruns]
    tau: np.ndarray   # float64 [nruns]
    rho0: np.ndarray  # float64 [sum N], runs concatenated
    steps: int

    @property
    def nruns(self) -> int:
        return int(self.N.size)

    @property
    def sites(self) -> int:
        return int(self.N.sum())

    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.N)])

    def run(self, r: int) -> np.ndarray:
        o = self.offsets()
        return self.rho0[o[r]:o[r + 1]]

    def subset(self, idx) -> "Workload":
        idx = np.asarray(idx)
        parts = [self.run(int(r)) for r in idx]
        return Workload(self.name + f"[{len(idx)} runs]", self.scheme, self.N[idx].copy(), self.L[idx].copy(),
                        self.dt[idx].copy(), self.tau[idx].copy(), np.concatenate(parts), self.steps)


def two_harmonic(N: int, L: float) -> np.ndarray:
    """cos(X/16)(1 + sin(X/16)) on X_j = j L / N."""
    X = np.arange(N) * (L / N)
    return np.cos(X / 16.0) * (1.0 + np.sin(X / 16.0))


def random_modes(N: int, L: float, rng: np.random.Generator, nmodes: int = 16, amp: float = 1e-2,
                 modes: np.ndarray | None = None) -> np.ndarray:
    """sum_m a_m cos(2 pi m X / L + phi_m), a_m ~ U(0, amp), phi_m ~ U(0, 2 pi);
    m = 1..nmodes unless given.  Zero mean by construction."""
    m = np.arange(1, nmodes + 1) if modes is None else np.asarray(modes)
    a = rng.uniform(0.0, amp, size=m.size)
    ph = rng.uniform(0.0, 2 * np.pi, size=m.size)
    X = np.arange(N) * (L / N)
    out = np.zeros(N)
    for mm, aa, pp in zip(m, a, ph):
        out += aa * np.cos(2 * np.pi * mm * X / L + pp)
    return out


def single_512() -> Workload:
    """D1Q5, N = 512 on L = 32 pi, two-harmonic field, tau = 1, dt = 5e-5, 10^4 steps."""
    L = 32 * np.pi
    return Workload("d1q5_n512_l32pi", 5, np.array([512]), np.array([L]), np.array([5e-5]), np.array([1.0]),
                    two_harmonic(512, L), 10_000)


def single_4096() -> Workload:
    """D1Q7, N = 4096 on L = 32 pi, two-harmonic field, tau = 3, dt = 5e-6 (to T = 150: 3e7 steps)."""
    L = 32 * np.pi
    return Workload("d1q7_n4096_l32pi", 7, np.array([4096]), np.array([L]), np.array([5e-6]), np.array([3.0]),
                    two_harmonic(4096, L), 30_000_000)


def ensemble(nruns: int = 4096, nmin: int = 256, nmax: int = 8192, dx: float = 0.1, dt: float = 1e-4,
             tau_range=(1.5, 3.0), steps: int = 100_000, seed: int = BASE_SEED) -> Workload:
    """D1Q7 ensemble: N log-uniform in [nmin, nmax], L = N dx, 16 random modes of
    amplitude U(0, 1e-2), tau ~ U(tau_range), one PCG64 stream per run."""
    Ns, taus, parts = [], [], []
    for r in range(nruns):
        rng = np.random.Generator(np.random.PCG64(seed + r))
        N = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        tau = float(rng.uniform(*tau_range))
        Ns.append(N)
        taus.append(tau)
        parts.append(random_modes(N, N * dx, rng))
    N = np.array(Ns, dtype=np.int64)
    return Workload(f"d1q7_ensemble_{nruns}x[{nmin},{nmax}]", 7, N, N * dx, np.full(nruns, dt), np.array(taus),
                    np.concatenate(parts), steps)


def ensemble_tau1(nruns: int = 4096, nmin: int = 256, nmax: int = 8192, dx: float = 0.2, dt: float = 5e-5,
                  steps: int = 100_000, seed: int = BASE_SEED) -> Workload:
    """The ensemble at tau = 1, the regime of the collapsed (rho-only) step:
    dx = 0.2 and dt = 5e-5, below the critical time step of the Sec. 3 fit at
    tau = 1 (7.2e-5 for D1Q7 at dx = 0.2).  Same lengths and modes as ensemble()."""
    wl = ensemble(nruns, nmin, nmax, dx, dt, (1.0, 1.0), steps, seed)
    return replace(wl, name=f"d1q7_ensemble_tau1_{nruns}x[{nmin},{nmax}]")


def long_lattice(N: int = 1 << 24, dx: float = 0.1, dt: float = 1e-4, tau: float = 1.51, nmodes: int = 64,
                 steps: int = 100_000, seed: int = BASE_SEED) -> Workload:
    """D1Q7 single lattice of N sites, 64 distinct modes m drawn from
    [1, floor(1.2 L / (2 pi))] (wavenumbers up to 1.2), amplitude U(0, 1e-2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = N * dx
    mmax = int(np.floor(1.2 * L / (2 * np.pi)))
    modes = rng.choice(np.arange(1, mmax + 1), size=nmodes, replace=False)
    a = rng.uniform(0.0, 1e-2, size=nmodes)
    ph = rng.uniform(0.0, 2 * np.pi, size=nmodes)
    X = np.arange(N) * dx
    rho = np.zeros(N)
    for mm, aa, pp in zip(modes, a, ph):
        rho += aa * np.cos(2 * np.pi * mm * X / L + pp)
    return Workload(f"d1q7_long_n{N}", 7, np.array([N], dtype=np.int64), np.array([L]), np.array([dt]),
                    np.array([tau]), rho, steps)


def chaos_ensemble(nruns: int = 1024, dt: float = 1e-4, tau: float = 3.0, steps: int = 1_000_000,
                   seed: int = BASE_SEED) -> Workload:
    """D1Q7 ensemble for long-time statistics: L ~ U(22, 200), dx log-uniform in
    [0.05, 0.1], N = round(L / dx), 16 random modes."""
    Ns, Ls, parts = [], [], []
    for r in range(nruns):
        rng = np.random.Generator(np.random.PCG64(seed + r))
        L = float(rng.uniform(22.0, 200.0))
        dx = float(np.exp(rng.uniform(np.log(0.05), np.log(0.1))))
        N = int(round(L / dx))
        Ns.append(N)
        Ls.append(L)
        parts.append(random_modes(N, L, rng))
    N = np.array(Ns, dtype=np.int64)
    return Workload(f"d1q7_chaos_{nruns}", 7, N, np.array(Ls), np.full(nruns, dt), np.full(nruns, tau),
                    np.concatenate(parts), steps)
