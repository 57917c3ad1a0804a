"""GPU solver parity: every solve must reach a true FP64 residual
|b - D x| / |b| <= 1e-10, recomputed here by the FP64 oracle on the returned
x (and by the GPU's own FP64 operator, reported in the stats).  The error
against the oracle's own CG solution is bounded by cond(D) * 1e-10 and is
checked loosely."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2001_05218_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dw():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_05218_gb300 import dw as m
    return m


def _resid(dims, kappa, U, x, b):
    return np.linalg.norm(O.dirac(dims, kappa, U, x) - b) / np.linalg.norm(b)


def test_small_workload_full_lattice_fp64(dw):
    dims, kappa, U, b = I.make_workload("wilson_4x4x4x4_haar")
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, b)
    x = dw.spinor(dims)
    s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner=dw.DW_F64, eo=0, verify_normal=1))
    xs = x.download()
    assert st[0]["true_rel_resid"] <= 1e-10
    assert _resid(dims, kappa, U, xs, b) <= 1e-10
    assert 0 < st[0]["normal_rel_resid"] < 1e-8
    xo, it, rr = O.cgnr(dims, kappa, U, b, tol=1e-12)
    assert np.linalg.norm(xs - xo) / np.linalg.norm(xo) < 1e-7
    # plain FP64 CGNR on both sides with the same stopping rule: iteration
    # counts agree up to rounding-order effects
    _, it10, _ = O.cgnr(dims, kappa, U, b, tol=1e-10)
    assert abs(st[0]["iters"] - it10) <= 2


@pytest.mark.parametrize("inner,c12,outer", [("f64", 0, "f64"), ("df64", 0, "f64"), ("f32", 0, "f64"),
                                            ("f32", 1, "df64"), ("f16", 1, "f64"), ("f16", 1, "df64"),
                                            ("bf16", 1, "df64"), ("f16", 0, "f64"), ("i16", 1, "df64"),
                                            ("i16", 0, "f64")])
@pytest.mark.parametrize("eo", [1, 0])
def test_mixed_solves_reach_fp64_residual(dw, inner, c12, outer, eo):
    dims, kappa = (8, 8, 8, 8), 0.122
    U = I.gauge_field(dims, "exp", 5, 1, 0.4)
    b = I.gaussian_spinor(dims, 5, 2)
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, b)
    x = dw.spinor(dims)
    s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner=inner, compress12=c12, eo=eo, outer=outer))
    assert s == dw.DW_OK
    assert st[0]["true_rel_resid"] <= 1e-10
    assert _resid(dims, kappa, U, x.download(), b) <= 1e-10
    if inner not in ("f64", "df64"):
        assert st[0]["reliable_updates"] >= 1


def test_medium_workload_eo_mixed_and_fp64(dw):
    dims, kappa, U, b = I.make_workload("wilson_16x16x16x32_exp0.4")
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, b)
    res = {}
    for inner, outer in (("f64", "f64"), ("f32", "f64"), ("f16", "df64")):
        x = dw.spinor(dims)
        s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner=inner, outer=outer,
                                                 compress12=1 if inner == "f16" else 0))
        assert s == dw.DW_OK and st[0]["true_rel_resid"] <= 1e-10
        xs = x.download()
        assert _resid(dims, kappa, U, xs, b) <= 1e-10
        res[inner] = (xs, st[0])
    # both solutions agree to the accuracy the residual bound allows
    for k in ("f32", "f16"):
        d = np.linalg.norm(res["f64"][0] - res[k][0]) / np.linalg.norm(res["f64"][0])
        assert d < 1e-7


MIXED = {"f32": dict(inner="f32"), "i16": dict(inner="i16", compress12=1, outer="df64")}


@pytest.mark.parametrize("inner", ["f32", "i16"])
def test_multi_rhs_point_sources(dw, inner):
    dims, kappa = (8, 8, 8, 16), 0.12
    U = I.gauge_field(dims, "exp", 8, 1, 0.4)
    srcs = np.stack([I.point_source(dims, s_, c_) for s_ in range(4) for c_ in range(3)])
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, srcs, nrhs=12)
    x = dw.spinor(dims, nrhs=12)
    s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, **MIXED[inner]))
    assert s == dw.DW_OK
    xs = x.download()
    for r in range(12):
        assert st[r]["true_rel_resid"] <= 1e-10
        assert _resid(dims, kappa, U, xs[r], srcs[r]) <= 1e-10


@pytest.mark.parametrize("inner", ["f32", "i16"])
def test_ragged_batch_of_lattices(dw, inner):
    systems = [((4, 4, 4, 4), 0.115), ((8, 4, 4, 8), 0.12), ((6, 6, 6, 6), 0.125), ((4, 4, 8, 8), 0.118)]
    Us, bs, xs, host = [], [], [], []
    for i, (dims, kappa) in enumerate(systems):
        U = I.gauge_field(dims, "exp", 40 + i, 1, 0.4)
        b = I.gaussian_spinor(dims, 40 + i, 2)
        Us.append(dw.gauge(dims, kappa, U))
        bs.append(dw.spinor(dims, b))
        xs.append(dw.spinor(dims))
        host.append((dims, kappa, U, b))
    s, st = dw.cg_solve_batched(Us, bs, xs, dw.params(tol=1e-10, **MIXED[inner]))
    assert s == dw.DW_OK
    for i, (dims, kappa, U, b) in enumerate(host):
        assert st[i]["true_rel_resid"] <= 1e-10
        assert _resid(dims, kappa, U, xs[i].download(), b) <= 1e-10


def test_normal_solve(dw):
    dims, kappa = (4, 4, 4, 8), 0.12
    U = I.gauge_field(dims, "exp", 9, 1, 0.4)
    b = I.gaussian_spinor(dims, 9, 2)
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, b)
    x = dw.spinor(dims)
    for outer in ("f64", "df64"):
        x = dw.spinor(dims)
        s, st = dw.cg_solve_normal(Ug, bg, x, dw.params(tol=1e-10, inner="f32", outer=outer))
        assert s == dw.DW_OK
        xs = x.download()
        r = np.linalg.norm(O.normal(dims, kappa, U, xs) - b) / np.linalg.norm(b)
        assert r <= 1e-10


def test_not_converged_and_bad_source(dw):
    dims, kappa = (4, 4, 4, 8), 0.12
    U = I.gauge_field(dims, "exp", 9, 1, 0.4)
    b = I.gaussian_spinor(dims, 9, 2)
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, b)
    x = dw.spinor(dims)
    s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, maxiter=3), raise_on_fail=False)
    assert s == dw.DW_ERR_NOT_CONVERGED and st[0]["iters"] <= 3 + 1
    bn = b.copy()
    bn[3, 1, 2] = np.nan
    bg2 = dw.spinor(dims, bn)
    s, st = dw.cg_solve(Ug, bg2, x, dw.params(tol=1e-10), raise_on_fail=False)
    assert s in (dw.DW_ERR_BREAKDOWN, dw.DW_ERR_NOT_CONVERGED)
    # the device-side time budget ends a solve with DW_ERR_TIMEOUT
    s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-14, inner="f32", timeout_s=1e-9, maxiter=100000),
                        raise_on_fail=False)
    assert s == dw.DW_ERR_TIMEOUT


@pytest.mark.parametrize("inner,delta", [("f32", 0.1), ("f16", 0.1), ("f32", 1e-3)])
def test_defect_correction_solves(dw, inner, delta):
    """The paper's two-data-type scheme: restarted low-precision inner CG,
    high-precision outer residual; reaches the same FP64 bound."""
    dims, kappa = (8, 8, 8, 16), 0.123
    U = I.gauge_field(dims, "exp", 12, 1, 0.4)
    b = I.gaussian_spinor(dims, 12, 2)
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, b)
    x = dw.spinor(dims)
    s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner=inner, delta=delta, defect_correction=1,
                                             outer="df64", compress12=1 if inner == "f16" else 0))
    assert s == dw.DW_OK and st[0]["reliable_updates"] >= 1
    assert _resid(dims, kappa, U, x.download(), b) <= 1e-10
