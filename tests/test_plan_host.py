"""CPU test of the resident kernel's planning (csrc/lbks_plan.h): compiles
tests/plan_check.cpp against the header with g++ and checks, on the benchmark
ensemble's lengths and on edge sets, that every site is stored by exactly one
piece, that pieces split into runs of S and S-1 sites per thread, that halves and
segments carry halos wide enough for the steps between exchanges, that groups hold
disjoint thread ranges within their capacity, that the segment-tree first fit
chooses the same group as a linear scan, that the counting sort ordering pieces
and bundles gives a stable sort's order, and that the plain kernel family's tiles
cover every site once at the tile size its rule picks.  No GPU needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "vector_types.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_check")
    subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Werror",
                    "-I" + os.path.join(ROOT, "paper_1711_03540_gb300", "csrc"),
                    "-I" + os.path.join(ROOT, "include"), "-I" + CUDA_INC,
                    os.path.join(ROOT, "tests", "plan_check.cpp"), "-o", exe], check=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True, timeout=300).stdout.splitlines()
        assert len(out) == len(lines)
        bad = [(l[:60], o) for l, o in zip(lines, out) if not o.startswith("OK")]
        assert not bad, bad
        return [dict(kv.split("=") for kv in o.split()[1:]) if "=" in o else {} for o in out]

    return run


def _line(C, S, NT, cl, kx, kseg, merge, Ns):
    return " ".join(str(int(v)) for v in (C, S, NT, cl, kx, kseg, merge, *Ns))


def _kseg(C, S, NT):
    return max(1, NT * S // (20 * C))


# (sites per thread, threads per block) of the resident kernel's tilings
TILINGS = ((12, 384), (8, 256), (16, 256), (6, 512), (4, 1024))


def test_benchmark_ensemble_plans(checker):
    from paper_1711_03540_gb300 import workloads

    Ns = workloads.ensemble(4096).N
    lines = []
    for S, NT in TILINGS:
        for merge in (0, 1):
            lines.append(_line(3, S, NT, 2, 32, _kseg(3, S, NT), merge, Ns))
    lines.append(_line(3, 12, 384, 1, 0, _kseg(3, 12, 384), 0, Ns))  # one-block groups: long runs segmented
    lines.append(_line(3, 12, 384, 2, 16, _kseg(3, 12, 384), 1, Ns))
    res = checker(lines)
    # 12 x 384: one block holds 4608 sites; every longer lattice is halved, and the
    # merged queue holds 1094 pair bundles (the benchmark's plan)
    assert int(res[1]["halves"]) == int((Ns > 12 * 384).sum()) == 687
    assert int(res[1]["blocks"]) == 0 and int(res[1]["segs"]) == 0 and int(res[1]["pairs"]) == 1094
    assert int(res[0]["blocks"]) > 0  # unmerged: single-block bundles keep their own queue
    assert int(res[10]["pairs"]) == 0 and int(res[10]["segs"]) > 0
    # packing: the groups' threads are mostly busy (rings 95-97 % with pairs, 99.5 %
    # with single blocks; a segment gets a block of its own)
    for j, d in enumerate(res):
        NT = TILINGS[j // 2][1] if j < 2 * len(TILINGS) else 384
        cap = (int(d["blocks"]) + 2 * int(d["pairs"])) * NT
        assert int(d["ring_threads"]) / cap > (0.98 if j == 10 else 0.94)
        if int(d["segblocks"]):
            assert int(d["seg_threads"]) / (int(d["segblocks"]) * NT) > 0.75


def test_edge_lengths(checker):
    rng = np.random.default_rng(7)
    S, NT = 4, 64
    cap = S * NT
    edges = [1, 2, 3, 7, S - 1, S, S + 1, cap - 1, cap, cap + 1, 2 * cap - 1, 2 * cap, 2 * cap + 1,
             3 * cap, 10 * cap + 3]
    lines = []
    for C in (2, 3):
        for cl, kx in ((1, 0), (2, 0), (2, 8), (2, 32)):
            for merge in (0, 1):
                lines.append(_line(C, S, NT, cl, kx, _kseg(C, S, NT), merge, edges))
                lines.append(_line(C, S, NT, cl, kx, 5, merge, rng.integers(1, 6 * cap, 300)))
    lines.append(_line(3, 16, 256, 2, 32, 40, 1, [1]))
    lines.append(_line(3, 8, 128, 1, 0, 1, 0, [1 << 20]))  # one long lattice in many segments
    lines.append(_line(2, 12, 384, 2, 32, 50, 1, rng.integers(200, 20000, 2000)))
    res = checker(lines)
    assert int(res[-2]["segs"]) >= (1 << 20) // (8 * 128)


def test_first_fit_matches_linear_scan(checker):
    checker(["FIRSTFIT 200 11", "FIRSTFIT 200 12"])


def test_counting_order_matches_stable_sort(checker):
    checker(["ORDER 200 21", "ORDER 200 22"])


def test_plain_family_tiles(checker):
    """The plain family's tiles cover every site once (reservoir lattices with their
    c_max ghosts on each side) and take the largest size of 256, 128, 64, 32 sites that
    gives each of 152 SMs two tiles: one 4096-site lattice (config 2) and one 512-site
    lattice (config 1) in 32-site tiles, the 4096-lattice ensemble in 256."""
    from paper_1711_03540_gb300 import workloads

    ens = workloads.ensemble(4096).N
    lines = ["PLAIN 152 0 3 4096", "PLAIN 152 0 2 512", "PLAIN 152 0 3 " + " ".join(map(str, ens)),
             "PLAIN 152 1 3 1201 601 301", "PLAIN 152 0 3 7", "PLAIN 152 1 2 5",
             "PLAIN 152 0 3 20000", "PLAIN 152 0 3 40000", "PLAIN 152 0 3 " + " ".join(["5000"] * 8),
             "PLAIN 152 0 3 " + " ".join(["300"] * 160), "PLAIN 152 0 3 " + " ".join(["64"] * 100)]
    res = checker(lines)
    assert res[0] == {"tile": "32", "tiles": "128"}
    assert res[1] == {"tile": "32", "tiles": "16"}
    assert res[2]["tile"] == "256"
    assert res[3] == {"tile": "32", "tiles": "67"}  # (1201 + 6) / 32 rounded up, and so on
    assert [r["tile"] for r in res[6:]] == ["64", "128", "128", "256", "32"]

