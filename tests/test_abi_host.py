"""CPU tests of the C ABI: the library loads and exports every entry point
declared in include/lb_ks.h, the binding's prototypes match the header's, the
host-side precompute matches the oracle, and argument validation fails cleanly
(no GPU needed)."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lb():
    from paper_1711_03540_gb300 import build

    build.build()
    import paper_1711_03540_gb300 as lb

    return lb


def _declared():
    txt = open(os.path.join(ROOT, "include", "lb_ks.h")).read()
    return sorted(set(re.findall(r"LB_KS_API[^;(]*?\b(lb_ks_\w+)\s*\(", txt)))


def test_header_declarations_exported(lb):
    import ctypes

    names = _declared()
    assert len(names) >= 15
    lib = ctypes.CDLL(lb.library_path())
    for n in names:
        assert hasattr(lib, n), f"{n} declared in lb_ks.h but not exported"
    assert sorted(lb.ABI_FUNCTIONS) == names  # the binding wraps exactly the declared ABI


@pytest.mark.parametrize("Q", [5, 7])
@pytest.mark.parametrize("alpha,beta,tau", [(0.1, 1e-4, 1.0), (0.2, 1e-3, 1.5), (0.0245, 5e-6, 3.0)])
@pytest.mark.parametrize("dmv", [0, 1, 2, 3])
def test_params_match_oracle(lb, Q, alpha, beta, tau, dmv):
    from oracle import lbks as ora

    A, B, coef = lb.lb_ks_params(Q, alpha, beta, tau, dmv)
    Ao, Bo = ora.feq_linear_quadratic(Q, alpha, beta, tau, dmv)
    np.testing.assert_allclose(A, Ao, rtol=1e-13, atol=1e-15)
    co = ora.coefficients(Q, alpha, beta, tau, dmv)
    # (feq(1) + feq(-1))/2 loses digits to cancellation; the oracle's J w1 does not
    w1 = ora.weight_full(1) if (Q == 7 and dmv & 2) else ora.weight(Q, 1)
    np.testing.assert_allclose(B, co["J"] * w1, rtol=1e-14, atol=0)
    np.testing.assert_allclose(B, Bo, rtol=0, atol=1e-14 * np.abs(Ao).max())
    np.testing.assert_allclose(coef, [co[k] for k in ["T1", "T2", "T3", "T4", "J", "K", "M", "dM", "E"]],
                               rtol=1e-13, atol=1e-300)
    # the equilibrium carries the mass: sum_i A_i = 1, sum_i B_i = 0
    assert abs(A.sum() - 1.0) < 1e-12 * max(1.0, np.abs(A).max())
    assert abs(B.sum()) < 1e-15


@pytest.mark.parametrize("Q", [5, 7])
@pytest.mark.parametrize("dmv", [0, 1, 2, 3])
def test_params_exact_pair_symmetry(lb, Q, dmv):
    """A_i is even and B_i odd in c_i exactly (bitwise, also after division by tau and
    rounding to FP32): the resident kernels take rho a_i and b_i of each -c plane from
    the +c plane before it."""
    import numpy as np

    for dx, dt, tau in [(0.1, 1e-4, 1.51), (0.2, 5e-5, 1.0), (0.0245, 5e-6, 3.0), (0.4, 2e-4, 2.7)]:
        A, B, _ = lb.lb_ks_params(Q, dx, dt, tau, dmv)
        for p in range(1, (Q - 1) // 2 + 1):
            assert A[2 * p] == A[2 * p - 1]
            assert B[2 * p] == -B[2 * p - 1]
            a, b = A / tau, B / tau
            assert a[2 * p] == a[2 * p - 1] and b[2 * p] == -b[2 * p - 1]
            assert np.float32(b[2 * p]) == -np.float32(b[2 * p - 1])


def test_params_reject_invalid(lb):
    for args in [(6, 0.1, 1e-4, 1.0), (7, 0.0, 1e-4, 1.0), (7, 0.1, -1.0, 1.0), (7, 0.1, 1e-4, 0.5),
                 (7, 0.1, 1e-4, math.nan)]:
        with pytest.raises(lb.LbKsError) as e:
            lb.lb_ks_params(*args)
        assert e.value.code == -1


def test_tau_fit_matches_oracle_and_paper(lb):
    from oracle import analysis

    for Q in (5, 7):
        for dX in (0.05, 0.1, 0.2):
            for dT in (1e-7, 1e-6, 1e-5, 1e-4, 1e-3):
                assert lb.lb_ks_tau_fit(Q, dX, dT) == pytest.approx(analysis.tau_fit(Q, dX, dT), rel=1e-13)
    assert lb.lb_ks_tau_fit(7, 0.1, 1e-4) == pytest.approx(1.5076, abs=1e-3)
    assert math.isnan(lb.lb_ks_tau_fit(4, 0.1, 1e-4))


@pytest.mark.parametrize("bad", [
    dict(scheme=6), dict(N=6), dict(L=0.0), dict(dt=-1e-4), dict(tau=0.95), dict(rho_nan=True),
    dict(opts=dict(precision=3)), dict(opts=dict(kernel=7)), dict(opts=dict(sites_per_thread=5)),
    dict(opts=dict(kernel=1, precision=2)), dict(opts=dict(threads_per_block=48)), dict(opts=dict(cluster_size=3)),
    dict(opts=dict(kernel=4)), dict(opts=dict(kernel=4, precision=2)),
])
def test_init_rejects_invalid_arguments(lb, bad):
    """Validation happens on the host before any device work: EINVAL on any
    machine (with or without a GPU), with a reason, and no handle."""
    args = dict(scheme=7, N=64, L=6.4, dt=1e-4, tau=1.5)
    args.update({k: v for k, v in bad.items() if k in args})
    rho0 = np.zeros(max(args["N"], 1))
    if bad.get("rho_nan"):
        rho0[3] = np.nan
    opts = lb.lb_ks_default_opts(**bad.get("opts", {}))
    with pytest.raises(lb.LbKsError) as e:
        lb.lb_ks_init(args["scheme"], args["N"], args["L"], args["dt"], args["tau"], rho0, opts)
    if bad.get("rho_nan"):
        assert e.value.code in (-1, -3)  # rho0 is read after the device check
    else:
        assert e.value.code == -1
    assert lb.lb_ks_last_error(None) not in ("", "no error")


@pytest.mark.parametrize("bad", [dict(kernel=2), dict(kernel=3), dict(recentre_every=10), dict(rho_left=np.nan)])
def test_reservoir_init_rejects_invalid_arguments(lb, bad):
    opts = lb.lb_ks_default_opts(**{k: v for k, v in bad.items() if k != "rho_left"})
    rl = bad.get("rho_left", 1.8)
    with pytest.raises(lb.LbKsError) as e:
        lb.lb_ks_batch_init_reservoir(7, [101], [60.0], [1e-4], [1.0], np.zeros(101), [rl], [4.2], opts)
    assert e.value.code == -1


def test_empty_batch_is_einval(lb):
    """An ensemble of no runs is EINVAL, checked on the host before any device work
    (periodic and reservoir constructors alike), with a reason and no handle."""
    e0 = np.zeros(0)
    with pytest.raises(lb.LbKsError) as e:
        lb.lb_ks_batch_init(7, np.zeros(0, dtype=np.int64), e0, e0, e0, e0)
    assert e.value.code == -1
    assert "nruns" in lb.lb_ks_last_error(None)
    with pytest.raises(lb.LbKsError) as e:
        lb.lb_ks_batch_init_reservoir(5, np.zeros(0, dtype=np.int64), e0, e0, e0, e0, e0, e0)
    assert e.value.code == -1


@pytest.mark.parametrize("Ns", [[(1 << 30) + 1], [1 << 30] * 17])
def test_size_limits_are_einval(lb, Ns):
    """A lattice above 2^30 sites, or more than 2^34 sites in all, is EINVAL before
    any device or host work on the lattices (rho0 is not read: a one-value buffer
    stands for it here)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("kept to machines where nothing could read past the one-value rho0")
    n = len(Ns)
    with pytest.raises(lb.LbKsError) as e:
        lb.lb_ks_batch_init(7, Ns, np.full(n, 1e8), np.full(n, 1e-4), np.full(n, 1.5), np.zeros(1))
    assert e.value.code == -1
    assert "2^3" in lb.lb_ks_last_error(None)


def test_no_device_is_an_error_not_a_fallback(lb):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lb.LbKsError) as e:
        lb.lb_ks_init(7, 64, 6.4, 1e-4, 1.5, np.zeros(64))
    assert e.value.code == -3


@pytest.mark.parametrize("Q", [5, 7])
@pytest.mark.parametrize("dx,dt,tau,rb", [(0.1, 1e-4, 1.5, 0.0), (0.1, 1e-4, 1.0, 0.0), (0.2, 5e-5, 1.0, 0.3),
                                          (0.05, 1e-5, 2.0, -0.5), (0.0245, 5e-6, 3.0, 0.0), (0.4, 1e-3, 1.2, 1.0)])
def test_max_growth_matches_oracle(lb, Q, dx, dt, tau, rb):
    """The library's characteristic-polynomial eigenvalues against the oracle's
    dense eigenvalue solver of the same amplification matrix."""
    from oracle import analysis

    g = lb.lb_ks_max_growth(Q, dx, dt, tau, rho_bar=rb, nk=64)
    ref = analysis.max_growth(Q, dx, dt, tau, rho_bars=(rb,), nk=64)
    assert g == pytest.approx(ref, rel=1e-6, abs=1e-6)


def test_max_growth_classifies_as_the_oracle_around_the_critical_step(lb):
    from oracle import analysis

    for Q, dx, tau in ((5, 0.1, 1.0), (7, 0.1, 1.0), (7, 0.2, 1.5)):
        dtc = analysis.critical_dt(Q, dx, tau)
        assert lb.lb_ks_max_growth(Q, dx, 0.9 * dtc, tau) <= 1.05 * 0.25
        assert lb.lb_ks_max_growth(Q, dx, 1.1 * dtc, tau) > 1.05 * 0.25
    with pytest.raises(lb.LbKsError):
        lb.lb_ks_max_growth(7, 0.1, 1e-4, 1.5, nk=0)


def _c_kind(t: str):
    """Kind and width of a C parameter or return type of lb_ks.h."""
    t = " ".join(t.replace("const", " ").split())
    if "*" in t:
        return "ptr"
    return {"void": None, "int": "i32", "int32_t": "i32", "uint32_t": "u32", "int64_t": "i64", "double": "f64",
            "size_t": "u64"}[t]


def _ctypes_kind(t):
    import ctypes as C

    if t is None:
        return None
    if t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer):
        return "ptr"
    if t is C.c_double:
        return "f64"
    if t is C.c_size_t:
        return "u64"
    if t is C.c_uint32:
        return "u32"
    return {4: "i32", 8: "i64"}[C.sizeof(t)]


def test_binding_prototypes_match_header(lb):
    """Every ctypes prototype of the binding has the header's return type and, parameter
    by parameter, the same kind and width (pointers as pointers)."""
    txt = re.sub(r"/\*.*?\*/", " ", open(os.path.join(ROOT, "include", "lb_ks.h")).read(), flags=re.S)
    protos = re.findall(r"LB_KS_API\s+([^;(]*?)\b(lb_ks_\w+)\s*\(([^)]*)\)\s*;", txt)
    assert len(protos) == len(lb.ABI_FUNCTIONS)
    for ret, name, params in protos:
        restype, argtypes = lb.ABI_FUNCTIONS[name]
        assert _ctypes_kind(restype) == _c_kind(ret), name
        c_params = []
        for prm in params.split(","):
            prm = " ".join(prm.split())
            typ = prm if "*" in prm else prm.rsplit(" ", 1)[0]  # drop the parameter's name
            c_params.append(_c_kind(typ))
        assert [_ctypes_kind(a) for a in argtypes] == c_params, name
