"""The second stencil behind the same solver: the gauge-covariant Laplacian
M = 1 - kappa K (spin-diagonal), dw_laplace_apply and dw_cg_solve_laplace
through the C ABI against the FP64 oracle (or_laplace, or_cg_laplace).

Operator bars as for the Wilson operator in the same storage: FP64 and
double-float 1e-13, FP32 1e-6, FP16 4e-3 per-site relative norm.  Solves:
true residual <= 1e-10 recomputed by the oracle, solution within 1e-8 of the
oracle's CG solution."""
import numpy as np
import pytest

from helpers import parity_of_sites, site_err
from oracle import oracle as O
from paper_2001_05218_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "df64": 1e-13, "f32": 1e-6, "f16": 4e-3}
DIMS = [(4, 4, 4, 6), (8, 6, 4, 10)]


@pytest.fixture(scope="module")
def dw():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_05218_gb300 import dw as m
    return m


def _schur_ref(dims, kappa, U, full, parity):
    """(1 - kappa^2 K_pq K_qp) psi_p from the oracle's full-lattice M."""
    par = parity_of_sites(dims)
    K = lambda v: (v - O.laplace(dims, kappa, U, v)) / kappa  # noqa: E731
    t = K(full)
    t[par == parity] = 0
    kt = K(t)
    return (full - kappa * kappa * kt)[par == parity]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec,c12", [("f64", 0), ("df64", 0), ("f32", 0), ("f32", 1), ("f16", 1), ("f16", 0)])
def test_laplace_apply_matches_oracle(dw, dims, prec, c12):
    kappa = 0.121
    U = I.gauge_field(dims, "haar", 51, 1, 0.5)
    psi = I.gaussian_spinor(dims, 51, 2)
    P = dw.PREC[prec]
    Ug = dw.gauge(dims, kappa, U, prec=P, compress12=c12)
    x, out = dw.spinor(dims, psi, prec=P), dw.spinor(dims, prec=P)
    dw.laplace_apply(Ug, x, out)
    assert site_err(out.download(), O.laplace(dims, kappa, U, psi)) <= TOL[prec]
    par = parity_of_sites(dims)
    for parity in (0, 1):
        kind = dw.DW_SPINOR_EVEN if parity == 0 else dw.DW_SPINOR_ODD
        full = np.where((par == parity)[:, None, None], psi, 0)
        xs = dw.spinor(dims, psi[par == parity], kind=kind, prec=P)
        os_ = dw.spinor(dims, kind=kind, prec=P)
        dw.laplace_apply(Ug, xs, os_)
        assert site_err(os_.download(), _schur_ref(dims, kappa, U, full, parity)) <= 10 * TOL[prec]


@pytest.mark.parametrize("inner,c12,outer", [("f64", 0, "f64"), ("f32", 0, "f64"), ("f32", 0, "df64"),
                                            ("f16", 1, "df64"), ("f16", 1, "f64")])
def test_laplace_solve_matches_oracle(dw, inner, c12, outer):
    dims, kappa = (8, 8, 8, 8), 0.1235
    U = I.gauge_field(dims, "exp", 53, 1, 0.4)
    b = I.gaussian_spinor(dims, 53, 2)
    Ug, bg, xg = dw.gauge(dims, kappa, U), dw.spinor(dims, b), dw.spinor(dims)
    s, st = dw.cg_solve_laplace(Ug, bg, xg, dw.params(tol=1e-10, inner=inner, compress12=c12, outer=outer))
    assert s == dw.DW_OK and st[0]["true_rel_resid"] <= 1e-10
    x = xg.download()
    assert np.linalg.norm(O.laplace(dims, kappa, U, x) - b) / np.linalg.norm(b) <= 1e-10
    xo, it, rr = O.cg_laplace(dims, kappa, U, b, tol=1e-13)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-8
    if inner != "f64":
        assert st[0]["reliable_updates"] >= 1


def test_laplace_multi_rhs_and_bad_precision(dw):
    dims, kappa, n = (4, 4, 4, 8), 0.12, 3
    U = I.gauge_field(dims, "exp", 55, 1, 0.4)
    bs = np.stack([I.gaussian_spinor(dims, 55, 2 + r) for r in range(n)])
    Ug, bg, xg = dw.gauge(dims, kappa, U), dw.spinor(dims, bs, nrhs=n), dw.spinor(dims, nrhs=n)
    s, st = dw.cg_solve_laplace(Ug, bg, xg, dw.params(tol=1e-10, inner="f16", compress12=1, outer="df64"))
    assert s == dw.DW_OK
    xs = xg.download()
    for r in range(n):
        assert np.linalg.norm(O.laplace(dims, kappa, U, xs[r]) - bs[r]) / np.linalg.norm(bs[r]) <= 1e-10
    s, _ = dw.cg_solve_laplace(Ug, bg, xg, dw.params(tol=1e-10, inner="bf16", compress12=1), raise_on_fail=False)
    assert s == dw.DW_ERR_PRECISION


def test_laplace_golden_fixture_on_gpu(dw):
    """The committed oracle fixture (extent-2 directions: forward and backward
    neighbours coincide) through dw_laplace_apply and dw_cg_solve_laplace."""
    from test_golden_and_inputs import load_golden_laplace
    meta, Mpsi, x = load_golden_laplace()
    dims, kappa, seed = meta["dims"], meta["kappa"], meta["seed"]
    U = I.gauge_field(dims, "haar", seed, 1)
    psi = I.gaussian_spinor(dims, seed, 2)
    Ug, pg, out = dw.gauge(dims, kappa, U), dw.spinor(dims, psi), dw.spinor(dims)
    dw.laplace_apply(Ug, pg, out)
    assert site_err(out.download(), Mpsi) <= 1e-13
    xg = dw.spinor(dims)
    s, st = dw.cg_solve_laplace(Ug, pg, xg, dw.params(tol=1e-12, inner="f64"))
    assert s == dw.DW_OK and np.linalg.norm(xg.download() - x) / np.linalg.norm(x) <= 1e-10
