"""Full-size workloads on the GPU, checked by the FP64 oracle at full size.

Each case runs in the configuration the benchmark uses (even-odd CGNR,
mixed precision, autotuned block shape, CUDA-graph loop) on the seeded
synthetic inputs of that workload, and the oracle recomputes the FP64 true
residual |b - D x| / |b| (or |b - D^dag D x| / |b|) on every site of the
returned solution: it must be <= 1e-10.  The full-size operator is also
compared with the oracle site by site."""
import numpy as np
import pytest

from helpers import site_err
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


@pytest.fixture(scope="module")
def big():
    return I.make_workload("wilson_32x32x32x64_exp0.6")


def test_bench_workload_operator_and_solve(dw, big):
    dims, kappa, U, b = big
    Ug = dw.gauge(dims, kappa, U)
    ref = O.dirac(dims, kappa, U, b)
    x = dw.spinor(dims, b)
    out = dw.spinor(dims)
    dw.apply(Ug, x, out)
    assert site_err(out.download(), ref) <= 1e-13
    del x, out
    bg = dw.spinor(dims, b)
    for inner, c12, outer in (("f16", 1, "df64"), ("f64", 0, "f64")):
        xg = dw.spinor(dims)
        s, st = dw.cg_solve(Ug, bg, xg, dw.params(tol=1e-10, inner=inner, compress12=c12, outer=outer))
        assert s == dw.DW_OK and st[0]["true_rel_resid"] <= 1e-10
        assert _resid(dims, kappa, U, xg.download(), b) <= 1e-10


def test_bench_workload_df64_operator(dw, big):
    dims, kappa, U, b = big
    Ug = dw.gauge(dims, kappa, U, prec=dw.DW_DF64)
    x = dw.spinor(dims, b, prec=dw.DW_DF64)
    out = dw.spinor(dims, prec=dw.DW_DF64)
    dw.apply(Ug, x, out)
    assert site_err(out.download(), O.dirac(dims, kappa, U, b)) <= 1e-13


def test_bench_workload_fp16_schur_operator(dw, big):
    """The operator the benchmark's solver iterates with, at full size: the
    FP16 (per-site scale, 16-bit operands, FP32 accumulation) even-site Schur
    complement with 12-real links, with the block shape the autotuner chose
    for this lattice (a solve first tunes it), site by site against the
    oracle, D and D^dag, and the reducing epilogue's FP64 |out|^2."""
    from helpers import parity_of_sites
    dims, kappa, U, b = big
    Ug = dw.gauge(dims, kappa, U)
    bg, xg = dw.spinor(dims, b), dw.spinor(dims)
    s, st = dw.cg_solve(Ug, bg, xg, dw.params(tol=1e-10, inner="f16", compress12=1, outer="df64"))
    assert s == dw.DW_OK
    del Ug, bg, xg
    par = parity_of_sites(dims)
    U16 = dw.gauge(dims, kappa, U, prec=dw.DW_F16, compress12=1)
    full = np.where((par == 0)[:, None, None], b, 0)
    x = dw.spinor(dims, b[par == 0], kind=dw.DW_SPINOR_EVEN, prec=dw.DW_F16)
    out = dw.spinor(dims, kind=dw.DW_SPINOR_EVEN, prec=dw.DW_F16)
    for dag in (False, True):
        n2 = dw.apply_norm(U16, x, out, dag=dag)
        ref = O.schur(dims, kappa, U, full, parity=0, dag=dag)[par == 0]
        assert site_err(out.download(), ref) <= 4e-3
        ref2 = float(np.vdot(ref.reshape(-1), ref.reshape(-1)).real)
        assert abs(n2[0] - ref2) <= 8e-3 * ref2
        dw.apply(U16, x, out, dag=dag)
        assert site_err(out.download(), ref) <= 4e-3


def test_medium_workload(dw):
    dims, kappa, U, b = I.make_workload("wilson_16x16x16x32_exp0.4")
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, b)
    for inner, outer in (("f32", "df64"), ("f32", "f64"), ("df64", "df64")):
        xg = dw.spinor(dims)
        s, st = dw.cg_solve(Ug, bg, xg, dw.params(tol=1e-10, inner=inner, outer=outer))
        assert s == dw.DW_OK
        assert _resid(dims, kappa, U, xg.download(), b) <= 1e-10


def test_twelve_point_sources_multi_rhs(dw):
    name = "wilson_24x24x24x48_exp0.4_12src"
    dims, kappa, U, _ = I.make_workload(name, with_source=False)
    srcs = np.stack([I.point_source(dims, s_, c_) for s_ in range(4) for c_ in range(3)])
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, srcs, nrhs=12)
    xg = dw.spinor(dims, nrhs=12)
    s, st = dw.cg_solve(Ug, bg, xg, dw.params(tol=1e-10, inner="f16", compress12=1, outer="df64"))
    assert s == dw.DW_OK
    xs = xg.download()
    for r in range(12):
        assert st[r]["true_rel_resid"] <= 1e-10
        assert _resid(dims, kappa, U, xs[r], srcs[r]) <= 1e-10


def test_ragged_batch_of_eight_lattices(dw):
    systems = I.ragged_batch()
    Us = [dw.gauge(d, k, U) for d, k, U, b in systems]
    bs = [dw.spinor(d, b) for d, k, U, b in systems]
    xs = [dw.spinor(d) for d, k, U, b in systems]
    s, st = dw.cg_solve_batched(Us, bs, xs, dw.params(tol=1e-10, inner="f16", compress12=1, outer="df64"))
    assert s == dw.DW_OK
    for i, (d, k, U, b) in enumerate(systems):
        assert st[i]["true_rel_resid"] <= 1e-10
        assert _resid(d, k, U, xs[i].download(), b) <= 1e-10


def test_gradient_workload(dw):
    import ctypes
    dims, kappa, U, b = I.make_workload("wilson_16x16x16x32_exp0.4_grad")
    g = I.gaussian_spinor(dims, I.workload_seed(4), I.STREAM_SOURCE2)
    Ug = dw.gauge(dims, kappa, U)
    bg, gx = dw.spinor(dims, b), dw.spinor(dims, g)
    gb, gU = dw.spinor(dims), dw.Field(Ug.lat, dw.DW_GAUGE)
    st = (dw.dw_solver_stats * 2)()
    p = dw.params(tol=1e-10, inner="f32", outer="df64")
    dw.check(dw.dw_cg_backward(Ug.handle, bg.handle, gx.handle, None, gb.handle, gU.handle, 0, ctypes.byref(p), st,
                               dw.current_stream()))
    lam = gb.download()
    # grad_b = (D^dag D)^{-1} g: residual of the adjoint solve, recomputed by the oracle
    r = np.linalg.norm(O.normal(dims, kappa, U, lam) - g) / np.linalg.norm(g)
    assert r <= 1e-10
    # forward solution and the force at sampled links, from the oracle's formula
    xg = dw.spinor(dims)
    dw.cg_solve_normal(Ug, bg, xg, p)
    x = xg.download()
    assert np.linalg.norm(O.normal(dims, kappa, U, x) - b) / np.linalg.norm(b) <= 1e-10
    Gref = O.force(dims, kappa, O.dirac(dims, kappa, U, x), lam) + O.force(dims, kappa, O.dirac(dims, kappa, U, lam), x)
    G = gU.download()
    rng = np.random.default_rng(11)
    idx = rng.integers(0, I.volume(dims), 64)
    # both sides use solves accurate to 1e-10: the force agrees to the solves' accuracy
    assert np.linalg.norm(G[idx] - Gref[idx]) / np.linalg.norm(Gref[idx]) < 1e-7
