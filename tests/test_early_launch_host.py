"""Source check of the programmatic dependent launch (no GPU needed).

The kernels that run one step per launch are launched with programmatic stream
serialisation (launch_early in csrc/lbks_device.cuh): their grid may be scheduled
while the previous step's grid still runs, which is correct only because every
thread first waits for that grid (wait_prior_grid) before it reads or writes global
memory: the previous step reads this step's destination and writes its source.  This
test finds every kernel passed to launch_early and checks that its body, or the device
function its body consists of, calls wait_prior_grid before its first access to the
kernel's global-memory parameters, so that a kernel added to that list without the
wait fails here instead of racing on the GPU."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1711_03540_gb300", "csrc")


def _sources():
    out = {}
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, name)) as f:
                out[name] = f.read()
    return out


def _body(src, name, kernel=True):
    """Text of the body of the function `name` (a __global__ kernel, or a device function)."""
    kind = r"__global__\s+void" if kernel else r"__device__\s+__forceinline__\s+void"
    m = re.search(kind + r"[^;{]*?\b" + re.escape(name) + r"\s*\(", src, re.S)
    if not m:
        return None
    i = src.index("{", m.end())
    depth, j = 0, i
    while True:
        c = src[j]
        depth += c == "{"
        depth -= c == "}"
        if depth == 0:
            return src[i + 1:j]
        j += 1


# global-memory parameters the step kernels read or write (tile list, run table, arenas)
_ACCESS = re.compile(r"\btiles\s*\[|\bruns\s*\[|\bsrc\.f\b|\bdst\.f\b")


def _waits_first(body):
    w = body.find("wait_prior_grid();")
    a = _ACCESS.search(body)
    return w >= 0 and (a is None or w < a.start())


def test_every_early_launched_kernel_waits_for_the_previous_grid_first():
    srcs = _sources()
    allsrc = "\n".join(srcs.values())
    launched = set()
    for text in srcs.values():
        launched.update(re.findall(r"launch_early\(\s*([A-Za-z_]\w*)\s*<", text))
    assert {"plain_step_kernel", "reservoir_step_kernel", "stream_step_kernel", "stream_step_kernel_f16",
            "collapse_step_kernel"} <= launched, launched
    for k in sorted(launched):
        body = _body(allsrc, k)
        assert body is not None, k
        if not _waits_first(body):
            # a thin entry whose body is one call of a device function: check that function
            calls = re.findall(r"\b([A-Za-z_]\w*)\s*<[^;]*>\s*\(", body)
            inner = [_body(allsrc, c, kernel=False) for c in calls]
            inner = [b for b in inner if b is not None]
            assert len(inner) == 1 and _waits_first(inner[0]), \
                f"{k} is launched early but does not wait for the previous grid before its first global access"


def test_the_check_catches_a_kernel_without_the_wait():
    """The same check on a planted kernel that reads its tiles before waiting."""
    src = """
template <int Q>
__global__ void planted_kernel(Arena src, Arena dst, const RunDesc* runs, const Tile* tiles) {
  const Tile tl = tiles[blockIdx.x];
  wait_prior_grid();
}
"""
    assert not _waits_first(_body(src, "planted_kernel"))
    good = src.replace("  const Tile tl = tiles[blockIdx.x];\n  wait_prior_grid();",
                       "  wait_prior_grid();\n  const Tile tl = tiles[blockIdx.x];")
    assert _waits_first(_body(good, "planted_kernel"))
