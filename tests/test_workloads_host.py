"""The seeded synthetic inputs hold the shapes and distributions stated for them:
the benchmark ensemble's lengths, relaxation times and zero-mean low-mode fields,
per-run seeding (a smaller ensemble is a prefix of a larger one, so subsets and
ranks see the same lattices), the long lattice's band-limited modes, and the
tau = 1 and long-time-statistics ensembles."""
import numpy as np
import pytest

from paper_1711_03540_gb300 import workloads


@pytest.fixture(scope="module")
def ens():
    return workloads.ensemble(4096)


def test_ensemble_lengths_log_uniform(ens):
    assert ens.nruns == 4096 and ens.scheme == 7
    assert ens.N.min() >= 256 and ens.N.max() <= 8192
    assert ens.sites == 9_379_578  # the benchmark's site count
    u = np.sort((np.log(ens.N) - np.log(256)) / (np.log(8192) - np.log(256)))
    ks = np.max(np.abs(u - (np.arange(1, u.size + 1) - 0.5) / u.size))  # Kolmogorov distance to U(0, 1)
    assert ks < 1.63 / np.sqrt(u.size)  # 1 % level
    np.testing.assert_allclose(ens.L, 0.1 * ens.N, rtol=1e-15)
    assert np.all(ens.dt == 1e-4) and ens.steps == 100_000


def test_ensemble_tau_and_fields(ens):
    assert ens.tau.min() >= 1.5 and ens.tau.max() < 3.0
    assert abs(np.mean(ens.tau) - 2.25) < 0.03
    off = ens.offsets()
    for r in range(0, ens.nruns, 97):
        x = ens.rho0[off[r]:off[r + 1]]
        assert abs(x.mean()) < 1e-15 and np.abs(x).max() <= 16 * 1e-2
        # only the modes m = 1..16 of the box: the spectrum is empty above them
        spec = np.abs(np.fft.rfft(x)) / x.size
        assert spec[17:].max() < 1e-15 and spec[1:17].max() > 1e-4 and spec[0] < 1e-15


def test_per_run_seeding_makes_prefixes(ens):
    small = workloads.ensemble(64)
    np.testing.assert_array_equal(small.N, ens.N[:64])
    np.testing.assert_array_equal(small.tau, ens.tau[:64])
    np.testing.assert_array_equal(small.rho0, ens.rho0[:small.sites])
    sub = ens.subset([5, 17])
    np.testing.assert_array_equal(sub.run(1), ens.run(17))


def test_tau1_ensemble_same_lattices_at_tau_1(ens):
    t1 = workloads.ensemble_tau1(256)
    np.testing.assert_array_equal(t1.N, ens.N[:256])
    assert np.all(t1.tau == 1.0) and np.all(t1.dt == 5e-5)
    np.testing.assert_allclose(t1.L, 0.2 * t1.N, rtol=1e-15)


def test_long_lattice_modes_in_the_ks_band():
    N = 1 << 16  # the generator's recipe at a size the host draws quickly
    wl = workloads.long_lattice(N=N)
    L = wl.L[0]
    spec = np.abs(np.fft.rfft(wl.rho0)) / N
    active = np.nonzero(spec > 1e-12)[0]
    assert active.size == 64
    assert active.min() >= 1 and active.max() <= np.floor(1.2 * L / (2 * np.pi))
    assert wl.tau[0] == 1.51 and wl.dt[0] == 1e-4 and abs(L / N - 0.1) < 1e-15


def test_chaos_ensemble_ranges():
    wl = workloads.chaos_ensemble(128)
    assert wl.L.min() >= 22.0 and wl.L.max() <= 200.0
    dx = wl.L / wl.N
    assert dx.min() > 0.05 * (1 - 1e-2) and dx.max() < 0.1 * (1 + 1e-2)
    assert np.all(wl.tau == 3.0) and np.all(wl.dt == 1e-4)


def test_two_harmonic_field():
    """cos(X/16)(1 + sin(X/16)) = cos(X/16) + sin(X/8)/2: on L = 32 pi exactly the
    modes m = 1 (cosine, amplitude 1) and m = 2 (sine, amplitude 1/2)."""
    x = workloads.two_harmonic(512, 32 * np.pi)
    c = np.fft.rfft(x) / 512
    np.testing.assert_allclose([c[1].real, c[1].imag, c[2].real, c[2].imag], [0.5, 0.0, 0.0, -0.25], atol=1e-15)
    c[1:3] = 0
    assert np.abs(c).max() < 1e-15
