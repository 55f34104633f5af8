"""CPU tests of bench.py: the reference arm (the FP64 oracle timed on the host
cores) prints one JSON line with the contract's keys, on the default arm's metric,
unit and workload, and under torchrun only rank 0 runs and prints; the clock
record of the timed region is read correctly from nvidia-smi's csv."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    p = _bench({}, "--impl", "reference", "--steps", "2", "--warmup", "3")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["metric"] == "lattice-site updates/s" and d["unit"] == "site-updates/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "d1q7_ensemble_4096x[256,8192]"
    assert d["config"]["nruns"] == 4096 and d["config"]["scheme"] == "D1Q7"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] > 0
    assert 1 <= cb["cores"] <= (os.cpu_count() or 1) and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    p = _bench({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, "--impl", "reference", "--gpus", "2",
               "--steps", "1", "--warmup", "3")
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_clock_sampler_reads_median_clock_and_active_reasons():
    """The clock record of the timed region: median SM clock over the samples, the
    maximum clock, and every throttle reason reported Active (csv, no units)."""
    sys.path.insert(0, ROOT)
    import bench

    class FinishedProcess:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.proc = FinishedProcess()
    cs.lines = [
        "2070, 2070, 901.25, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1965, 2070, 1391.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1203.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",  # a sample the driver could not read
        "",
    ]
    r = cs.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    cs.lines = ["1400, 2070, 1000.0, 0x0000000000000008, Active, Not Active, Active, Not Active"]
    r = cs.stop()
    assert r["sm_mhz"] == 1400.0 and r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
