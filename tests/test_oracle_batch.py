"""Pin of the oracle's ensemble entry point (lbo_run_batch, oracle/lbks.py run_batch).

run_batch is the checker of every ensemble parity test: it slices the concatenated
rho0 and the per-run N, alpha, beta, tau and spreads the runs over OpenMP threads.
Each run of a batch is an independent periodic lattice of the scheme of Sec. 2
(Eq. LB_equation_ordinary), so its result is fixed by the single-run entry point
lbo_run on that run alone.  These tests require bitwise equality with it, for one
and for many threads, on ragged batches whose runs differ in every parameter, so
that an offset, a parameter mix-up or a run computed twice fails them.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import lbks as ora


def _batch(Q: int, seed: int):
    cmax = (Q - 1) // 2
    rng = np.random.default_rng(seed)
    # minimum lattice, primes, a power of two, and lengths around it
    Ns = np.array([2 * cmax + 1, 13, 97, 251, 256, 257, 1009, 2 * cmax + 2], dtype=np.int64)
    k = Ns.size
    alpha = rng.uniform(0.08, 0.3, k)
    beta = rng.uniform(2e-5, 1e-4, k)
    tau = rng.uniform(1.0, 3.0, k)
    rho0 = np.concatenate([0.1 * rng.standard_normal(n) + rng.uniform(-0.2, 0.2) for n in Ns])
    return Ns, alpha, beta, tau, rho0


def _per_run(Q, Ns, alpha, beta, tau, rho0, n, dm_variant=ora.DM_DERIVED):
    off = np.concatenate([[0], np.cumsum(Ns)])
    return np.concatenate([ora.run(Q, rho0[off[r]:off[r + 1]], alpha[r], beta[r], tau[r], n, dm_variant=dm_variant)
                           for r in range(Ns.size)])


@pytest.mark.parametrize("Q", [5, 7])
@pytest.mark.parametrize("nthreads", [1, 16])
def test_batch_equals_single_runs_bitwise(Q, nthreads):
    Ns, alpha, beta, tau, rho0 = _batch(Q, 100 + Q)
    n = 150
    got, used = ora.run_batch(Q, Ns, alpha, beta, tau, rho0, n, nthreads=nthreads)
    assert 1 <= used <= nthreads
    np.testing.assert_array_equal(got, _per_run(Q, Ns, alpha, beta, tau, rho0, n))


def test_batch_printed_delta_m_reading_equals_single_runs():
    Q = 7
    Ns, alpha, beta, tau, rho0 = _batch(Q, 7)
    n = 80
    got, _ = ora.run_batch(Q, Ns, alpha, beta, tau, rho0, n, dm_variant=ora.DM_PRINTED, nthreads=4)
    np.testing.assert_array_equal(got, _per_run(Q, Ns, alpha, beta, tau, rho0, n, dm_variant=ora.DM_PRINTED))


def test_batch_comparison_detects_a_parameter_mixup():
    """The comparison above is sharp: two runs' tau (or their rho0 slices) exchanged
    change the batch's result."""
    Q = 7
    Ns, alpha, beta, tau, rho0 = _batch(Q, 3)
    n = 60
    ref = _per_run(Q, Ns, alpha, beta, tau, rho0, n)
    tau_x = tau.copy()
    tau_x[[2, 3]] = tau_x[[3, 2]]
    got, _ = ora.run_batch(Q, Ns, alpha, beta, tau_x, rho0, n, nthreads=2)
    assert not np.array_equal(got, ref)
    # runs 4 and 5 have 256 and 257 sites: shifting the slice by one site moves every value
    off = np.concatenate([[0], np.cumsum(Ns)])
    r0 = rho0.copy()
    r0[off[4]:off[5]] = rho0[off[4] + 1:off[5] + 1]
    got, _ = ora.run_batch(Q, Ns, alpha, beta, tau, r0, n, nthreads=2)
    assert not np.array_equal(got[off[4]:off[5]], ref[off[4]:off[5]])


def test_batch_of_zero_steps_returns_rho0():
    Q = 5
    Ns, alpha, beta, tau, rho0 = _batch(Q, 11)
    got, _ = ora.run_batch(Q, Ns, alpha, beta, tau, rho0, 0, nthreads=3)
    # f = f^eq(rho0) sums back to rho0 up to the rounding of the equilibrium's terms
    assert np.max(np.abs(got - rho0)) <= 1e-15 * max(1.0, np.abs(rho0).max()) * 8
