"""Long-time statistics of chaotic Kuramoto-Sivashinsky ensembles, for comparing
storage precisions where trajectories cannot be compared point by point.

For every run of a batched handle: the time average of <rho^2> = (1/N) sum_x rho^2
(from the FP64 energy reduction of lb_ks_mass_energy) and the time-averaged energy
spectrum |rho_k|^2 (numpy FFT of lb_ks_rho snapshots), averaged over the ensemble
in wavenumber bins (the runs have different lengths L, so k = 2 pi m / L differs).
Averages start after a burn-in.  Sec. 1 motivates KS as a model of spatio-temporal
chaos; the statistics are those any KS study reports.

    python -m paper_1711_03540_gb300.chaos --steps 1000000 --burn-in 200000

runs the 1024-run chaos ensemble in FP32 and in scaled FP16 (with the FP64 guard)
and in FP64 and prints one JSON line with the statistics and the relative
differences of each reduced storage against FP64.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

K_BINS = np.linspace(0.0, 1.5, 31)  # KS is driven below k = 1; 0.05-wide bins


def ensemble_statistics(wl, precision: int, steps: int, burn_in: int, sample_every: int = 1000,
                        spectrum_every: int = 10_000, recentre_every: int = 500, kernel: int = 0, k_bins=K_BINS,
                        stream=None) -> dict:
    """Advance the workload's runs `steps` steps; average over samples taken every
    sample_every (energy) / spectrum_every (spectrum) steps after `burn_in` steps."""
    from . import (F64, lb_ks_batch_init, lb_ks_default_opts, lb_ks_free, lb_ks_mass_energy, lb_ks_rho,
                   lb_ks_step)

    if steps % sample_every or burn_in % sample_every or spectrum_every % sample_every:
        raise ValueError("steps, burn_in and spectrum_every must be multiples of sample_every")
    opts = lb_ks_default_opts(precision=precision, kernel=kernel,
                              recentre_every=0 if precision == F64 else recentre_every, stream=stream)
    t0 = time.perf_counter()
    h = lb_ks_batch_init(wl.scheme, wl.N, wl.L, wl.dt, wl.tau, wl.rho0, opts)
    nruns = int(wl.N.size)
    off = np.concatenate([[0], np.cumsum(wl.N)])
    energy = np.empty(nruns)
    rho = np.empty(int(wl.N.sum()))
    e_sum = np.zeros(nruns)
    n_e = 0
    nb = len(k_bins) - 1
    spec = np.zeros(nb)
    n_s = 0
    try:
        done = 0
        while done < steps:
            lb_ks_step(h, sample_every)
            done += sample_every
            if done <= burn_in:
                continue
            lb_ks_mass_energy(h, None, energy)
            e_sum += energy / wl.N
            n_e += 1
            if done % spectrum_every == 0:
                lb_ks_rho(h, rho)
                spec += _binned_spectrum(rho, off, wl.L, k_bins)
                n_s += 1
    finally:
        lb_ks_free(h)
    seconds = time.perf_counter() - t0
    return {"mean_rho2": e_sum / max(n_e, 1), "spectrum": spec / max(n_s, 1), "k_bins": np.asarray(k_bins),
            "energy_samples": n_e, "spectrum_samples": n_s, "seconds": seconds,
            "site_updates": float(wl.N.sum()) * steps}


def _binned_spectrum(rho, off, L, k_bins) -> np.ndarray:
    """Ensemble-mean spectral density in k bins: for each run, 2 |rho_m|^2 (m >= 1,
    rho_m the Fourier coefficients, so that sum_m 2|rho_m|^2 is the variance of rho)
    summed over the modes k = 2 pi m / L that fall in a bin and divided by the bin
    width (so the density integrates to the variance, whatever L), then averaged over
    runs."""
    nb = len(k_bins) - 1
    out = np.zeros(nb)
    dk = np.diff(k_bins)
    for r in range(len(off) - 1):
        x = rho[off[r]:off[r + 1]]
        n = x.size
        c = np.fft.rfft(x) / n
        m = np.arange(1, c.size)
        p = 2.0 * np.abs(c[1:]) ** 2
        if n % 2 == 0:
            p[-1] *= 0.5  # the Nyquist coefficient has no mirror
        k = 2.0 * np.pi * m / L[r]
        idx = np.searchsorted(k_bins, k, side="right") - 1
        ok = (idx >= 0) & (idx < nb)
        out += np.bincount(idx[ok], weights=p[ok], minlength=nb) / dk
    return out / (len(off) - 1)


def compare(a: dict, b: dict, rel_floor: float = 0.01) -> dict:
    """Relative differences of b against a: ensemble-mean <rho^2>, and the spectrum
    in the bins holding at least rel_floor of a's largest bin."""
    m_a, m_b = float(np.mean(a["mean_rho2"])), float(np.mean(b["mean_rho2"]))
    sa, sb = a["spectrum"], b["spectrum"]
    sel = sa >= rel_floor * sa.max()
    return {"mean_rho2_rel": abs(m_b - m_a) / m_a,
            "spectrum_max_rel": float(np.max(np.abs(sb[sel] - sa[sel]) / sa[sel])),
            "bins_compared": int(sel.sum())}


def main() -> None:
    from . import F16S, F32, F64, build, workloads

    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--nruns", type=int, default=1024)
    p.add_argument("--steps", type=int, default=1_000_000)
    p.add_argument("--burn-in", type=int, default=200_000)
    args = p.parse_args()
    build.build()
    wl = workloads.chaos_ensemble(nruns=args.nruns)
    s32 = ensemble_statistics(wl, F32, args.steps, args.burn_in)
    s16 = ensemble_statistics(wl, F16S, args.steps, args.burn_in)
    s64 = ensemble_statistics(wl, F64, args.steps, args.burn_in)
    cmp = compare(s64, s32)
    line = {"workload": wl.name, "sites": int(wl.N.sum()), "steps": args.steps, "burn_in": args.burn_in,
            "dt": float(wl.dt[0]), "T": args.steps * float(wl.dt[0]),
            "fp32": {"mean_rho2": float(np.mean(s32["mean_rho2"])), "seconds": s32["seconds"],
                     "site_updates_per_s": s32["site_updates"] / s32["seconds"]},
            "fp64": {"mean_rho2": float(np.mean(s64["mean_rho2"])), "seconds": s64["seconds"],
                     "site_updates_per_s": s64["site_updates"] / s64["seconds"]},
            "f16s": {"mean_rho2": float(np.mean(s16["mean_rho2"])), "seconds": s16["seconds"],
                     "site_updates_per_s": s16["site_updates"] / s16["seconds"]},
            "fp32_vs_fp64": cmp,
            "f16s_vs_fp64": compare(s64, s16),
            "spectrum_f16s": [float(v) for v in s16["spectrum"]],
            "spectrum_fp64": [float(v) for v in s64["spectrum"]],
            "spectrum_fp32": [float(v) for v in s32["spectrum"]],
            "k_bins": [float(v) for v in K_BINS]}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
