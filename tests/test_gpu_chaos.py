"""Long-time statistics of the chaotic D1Q7 ensemble (1024 runs, L ~ U(22, 200),
Delta X log-uniform in [0.05, 0.1], tau = 3, Delta T = 1e-4): FP32 and scaled-FP16
storage with the FP64 guard against FP64, by the ensemble-mean time-averaged <rho^2>
and the time-averaged energy spectrum in wavenumber bins, each within 2 % (bins
holding at least 1 % of the largest).  Trajectories of a chaotic system are compared
by statistics, not point by point.  This test runs T = 30 with averages over
T in (10, 30]; `python -m paper_1711_03540_gb300.chaos` runs the full T = 100
with a T = 20 burn-in."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03540_gb300 import build

    build.build()
    import paper_1711_03540_gb300 as lb

    return lb


STEPS, BURN = 300_000, 100_000


@pytest.fixture(scope="module")
def fp64_statistics(lb):
    from paper_1711_03540_gb300 import chaos, workloads

    wl = workloads.chaos_ensemble(nruns=1024)
    s64 = chaos.ensemble_statistics(wl, lb.F64, STEPS, BURN)
    assert s64["energy_samples"] == 200 and s64["spectrum_samples"] == 20
    assert np.all(np.isfinite(s64["mean_rho2"])) and np.mean(s64["mean_rho2"]) > 1e-3  # the runs are active
    return wl, s64


@pytest.mark.parametrize("prec", ["F32", "F16S"])
def test_reduced_storage_statistics_match_fp64(lb, fp64_statistics, prec):
    from paper_1711_03540_gb300 import chaos

    wl, s64 = fp64_statistics
    s = chaos.ensemble_statistics(wl, getattr(lb, prec), STEPS, BURN)
    c = chaos.compare(s64, s)
    assert c["bins_compared"] >= 10
    assert c["mean_rho2_rel"] <= 0.02, c
    assert c["spectrum_max_rel"] <= 0.02, c
