"""CPU tests of the long-time statistics helpers (paper_1711_03540_gb300.chaos):
the binned spectral density integrates to the variance (Parseval) and puts a pure
mode in the bin of its wavenumber, whatever the lattice length."""
import numpy as np
import pytest

from paper_1711_03540_gb300 import chaos


def test_pure_mode_lands_in_its_bin_and_integrates_to_its_variance():
    a, m0 = 0.3, 5
    rows, Ls = [], []
    for n, L in ((256, 20 * np.pi), (200, 40 * np.pi)):
        x = np.arange(n) * (L / n)
        mm = m0 * int(round(L / (20 * np.pi)))  # the same k = 0.5 in both runs
        rows.append(0.7 + a * np.cos(2 * np.pi * mm * x / L + 0.4))
        Ls.append(L)
    off = np.array([0, 256, 456])
    spec = chaos._binned_spectrum(np.concatenate(rows), off, np.array(Ls), chaos.K_BINS)
    dk = np.diff(chaos.K_BINS)
    assert (spec * dk).sum() == pytest.approx(a * a / 2, rel=1e-12)
    b = np.searchsorted(chaos.K_BINS, 0.5, side="right") - 1
    assert spec[b] * dk[b] == pytest.approx(a * a / 2, rel=1e-12)
    assert np.count_nonzero(spec > 1e-20) == 1


def test_parseval_on_random_fields():
    rng = np.random.default_rng(0)
    n, L = 512, 51.2
    x = rng.standard_normal(n)
    spec = chaos._binned_spectrum(x, np.array([0, n]), np.array([L]), np.linspace(0, 2 * np.pi * n / L, 200))
    dk = 2 * np.pi * n / L / 199
    assert (spec * dk).sum() == pytest.approx(np.var(x), rel=1e-10)


def test_compare():
    a = {"mean_rho2": np.array([1.0, 1.0]), "spectrum": np.array([1.0, 0.5, 1e-4])}
    b = {"mean_rho2": np.array([1.01, 1.01]), "spectrum": np.array([1.02, 0.49, 5.0])}
    c = chaos.compare(a, b)
    assert c["mean_rho2_rel"] == pytest.approx(0.01)
    assert c["spectrum_max_rel"] == pytest.approx(0.02)  # the bin below 1 % of the peak is not compared
    assert c["bins_compared"] == 2
