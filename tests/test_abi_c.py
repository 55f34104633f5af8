"""The C ABI from C: tests/abi_check.c, compiled as C11 with -pedantic -Werror
against include/lb_ks.h and linked to the library, runs its checks (host
precompute, argument errors, NULL handles; without a device, LB_KS_ECUDA from
the constructors; with one, a short run), and its layout mode shows that the
Python binding's options struct and constants are the header's."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc is missing")
    from paper_1711_03540_gb300 import build

    build.build()
    import paper_1711_03540_gb300 as lb

    lib = lb.library_path()
    path = str(tmp_path_factory.mktemp("abi") / "abi_check")
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-O1",
                    "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_check.c"), lib,
                    "-Wl,-rpath," + os.path.dirname(lib), "-lm", "-o", path], check=True)
    return path


def test_c_caller(exe):
    p = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    lines = p.stdout.splitlines()
    assert p.returncode == 0 and lines and all(ln.startswith("OK") for ln in lines), p.stdout + p.stderr
    assert len(lines) >= 9


def test_binding_matches_header_layout(exe):
    import paper_1711_03540_gb300 as lb

    p = subprocess.run([exe, "layout"], capture_output=True, text=True, timeout=60, check=True)
    out = {k: int(v) for k, v in (ln.split() for ln in p.stdout.splitlines())}
    # lb_ks_opts: same fields, offsets and size as the ctypes structure
    assert out["sizeof_opts"] == C.sizeof(lb.LbKsOpts)
    c_fields = {k[len("offset_"):] for k in out if k.startswith("offset_")}
    assert c_fields == {name for name, _ in lb.LbKsOpts._fields_}
    for name, _ in lb.LbKsOpts._fields_:
        assert out["offset_" + name] == getattr(lb.LbKsOpts, name).offset, name
    # constants
    binding = {"LB_KS_D1Q5": lb.D1Q5, "LB_KS_D1Q7": lb.D1Q7, "LB_KS_F64": lb.F64, "LB_KS_F32": lb.F32,
               "LB_KS_F16S": lb.F16S, "LB_KS_KERNEL_AUTO": lb.KERNEL_AUTO, "LB_KS_KERNEL_PLAIN": lb.KERNEL_PLAIN,
               "LB_KS_KERNEL_STREAM": lb.KERNEL_STREAM, "LB_KS_KERNEL_RESIDENT": lb.KERNEL_RESIDENT,
               "LB_KS_KERNEL_COLLAPSE": lb.KERNEL_COLLAPSE, "LB_KS_DM_DERIVED": lb.DM_DERIVED,
               "LB_KS_DM_PRINTED": lb.DM_PRINTED, "LB_KS_WEIGHTS_FULL_INVERSE": lb.WEIGHTS_FULL_INVERSE,
               "LB_KS_LANE_FIELDS": len(lb.LANE_FIELDS)}
    for k, v in binding.items():
        assert out[k] == v, k
    statuses = {k for k in out if k == "LB_KS_OK" or k.startswith("LB_KS_E")}
    assert statuses == set(lb.STATUS.values())
    for code, name in lb.STATUS.items():
        assert out[name] == code, name
