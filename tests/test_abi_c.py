"""The C ABI from C: tests/abi_check.c, compiled as C11 with -pedantic -Werror
against include/lb_ks.h and linked to the library, runs its checks (host
precompute, argument errors, NULL handles; without a device, LB_KS_ECUDA from
the constructors; with one, a short run)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_caller(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc is missing")
    from paper_1711_03540_gb300 import build

    build.build()
    import paper_1711_03540_gb300 as lb

    lib = lb.library_path()
    exe = str(tmp_path / "abi_check")
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-O1",
                    "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_check.c"), lib,
                    "-Wl,-rpath," + os.path.dirname(lib), "-lm", "-o", exe], check=True)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    lines = p.stdout.splitlines()
    assert p.returncode == 0 and lines and all(ln.startswith("OK") for ln in lines), p.stdout + p.stderr
    assert len(lines) >= 9
