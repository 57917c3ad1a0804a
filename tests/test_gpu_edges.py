"""Edge cases of the GPU path: extreme lattice shapes, batches beyond one
launch, plan-cache reuse and eviction, converged starting guesses, optional
diagnostics -- each checked against the FP64 oracle."""
import numpy as np
import pytest

from helpers import parity_of_sites, site_err
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


@pytest.mark.parametrize("dims", [(2, 4, 4, 4), (2, 2, 2, 8), (4, 2, 2, 2), (12, 2, 6, 4)])
def test_thin_lattices_apply_and_solve(dw, dims):
    """Extent 2 in a direction: forward and backward neighbours coincide (and
    Lx = 2 gives a half extent of 1 for the even-odd index)."""
    kappa = 0.12
    U = I.gauge_field(dims, "haar", 81, 1)
    b = I.gaussian_spinor(dims, 81, 2)
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, b)
    out = dw.spinor(dims)
    for dag in (False, True):
        dw.apply(Ug, bg, out, dag=dag)
        assert site_err(out.download(), O.dirac(dims, kappa, U, b, dag=dag)) <= 1e-13
    for inner in ("f64", "f32"):
        x = dw.spinor(dims)
        s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner=inner, outer="df64"))
        assert s == dw.DW_OK and _resid(dims, kappa, U, x.download(), b) <= 1e-10


def test_batch_larger_than_one_launch(dw):
    """More systems than one launch holds: the batch is split into launches."""
    systems = []
    for i in range(11):
        dims = [(4, 4, 4, 4), (4, 4, 2, 8), (6, 4, 4, 4)][i % 3]
        kappa = 0.11 + 0.002 * i
        systems.append((dims, kappa, I.gauge_field(dims, "exp", 90 + i, 1, 0.4), I.gaussian_spinor(dims, 90 + i, 2)))
    Us = [dw.gauge(d, k, U) for d, k, U, b in systems]
    bs = [dw.spinor(d, b) for d, k, U, b in systems]
    xs = [dw.spinor(d) for d, k, U, b in systems]
    s, st = dw.cg_solve_batched(Us, bs, xs, dw.params(tol=1e-10, inner="f32"))
    assert s == dw.DW_OK and len(st) == 11
    for i, (d, k, U, b) in enumerate(systems):
        assert st[i]["true_rel_resid"] <= 1e-10
        assert _resid(d, k, U, xs[i].download(), b) <= 1e-10


def test_plan_cache_reuse_and_eviction(dw):
    """Repeated solves of the same fields reuse the cached plan and graph; more
    distinct problems than the cache holds evict older plans; every solve stays
    correct and repeatable (bitwise, deterministic reductions)."""
    dims, kappa = (4, 4, 4, 8), 0.12
    U = I.gauge_field(dims, "exp", 95, 1, 0.4)
    Ug = dw.gauge(dims, kappa, U)
    sols = []
    for rep in range(2):
        for k in range(6):  # six different (b, x) pairs -> six plans
            b = I.gaussian_spinor(dims, 95, 10 + k)
            bg, x = dw.spinor(dims, b), dw.spinor(dims)
            s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner="f16", compress12=1, outer="df64"))
            assert s == dw.DW_OK
            xs = x.download()
            assert _resid(dims, kappa, U, xs, b) <= 1e-10
            if rep == 0:
                sols.append(xs)
            else:
                assert np.array_equal(xs, sols[k])
    # the same fields solved twice in a row through the cached graph
    b = I.gaussian_spinor(dims, 95, 40)
    bg, x = dw.spinor(dims, b), dw.spinor(dims)
    p = dw.params(tol=1e-10, inner="f32", outer="df64")
    dw.cg_solve(Ug, bg, x, p)
    x1 = x.download()
    x.storage.zero_()
    dw.cg_solve(Ug, bg, x, p)
    assert np.array_equal(x1, x.download())


def test_converged_guess_and_zero_source(dw):
    dims, kappa = (4, 4, 4, 8), 0.12
    U = I.gauge_field(dims, "exp", 96, 1, 0.4)
    b = I.gaussian_spinor(dims, 96, 2)
    Ug, bg = dw.gauge(dims, kappa, U), dw.spinor(dims, b)
    x = dw.spinor(dims)
    dw.cg_solve(Ug, bg, x, dw.params(tol=1e-12, inner="f64"))
    s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner="f32", outer="df64"))
    assert s == dw.DW_OK and st[0]["iters"] <= 1
    zero = dw.spinor(dims)
    x2 = dw.spinor(dims, b)  # non-zero guess, zero source: the solution is 0
    s, st = dw.cg_solve(Ug, zero, x2, dw.params(tol=1e-10, inner="f32"))
    assert s == dw.DW_OK
    assert np.abs(x2.download()).max() < 1e-9


def test_nonzero_initial_guess(dw):
    dims, kappa = (6, 4, 4, 8), 0.121
    U = I.gauge_field(dims, "exp", 97, 1, 0.4)
    b = I.gaussian_spinor(dims, 97, 2)
    g0 = I.gaussian_spinor(dims, 97, 3)
    Ug, bg = dw.gauge(dims, kappa, U), dw.spinor(dims, b)
    for eo in (1, 0):
        for outer in ("f64", "df64"):
            x = dw.spinor(dims, g0)
            s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner="f16", compress12=1, outer=outer, eo=eo))
            assert s == dw.DW_OK and _resid(dims, kappa, U, x.download(), b) <= 1e-10


def test_verify_normal_with_double_float_outer(dw):
    dims, kappa = (4, 4, 4, 8), 0.12
    U = I.gauge_field(dims, "exp", 98, 1, 0.4)
    b = I.gaussian_spinor(dims, 98, 2)
    Ug, bg = dw.gauge(dims, kappa, U), dw.spinor(dims, b)
    x = dw.spinor(dims)
    s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner="f32", outer="df64", verify_normal=1))
    xs = x.download()
    r = b - O.dirac(dims, kappa, U, xs)
    expect = np.linalg.norm(O.dirac(dims, kappa, U, r, dag=True)) / np.linalg.norm(O.dirac(dims, kappa, U, b, dag=True))
    assert abs(st[0]["normal_rel_resid"] - expect) <= 1e-3 * expect + 1e-16


def test_bf16_multi_rhs_solve(dw):
    dims, kappa = (8, 4, 4, 8), 0.118
    U = I.gauge_field(dims, "exp", 99, 1, 0.4)
    bs = np.stack([I.gaussian_spinor(dims, 99, 10 + r) for r in range(6)])
    Ug = dw.gauge(dims, kappa, U)
    bg, x = dw.spinor(dims, bs, nrhs=6), dw.spinor(dims, nrhs=6)
    s, st = dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner="bf16", compress12=1, outer="df64"))
    assert s == dw.DW_OK
    xs = x.download()
    for r in range(6):
        assert _resid(dims, kappa, U, xs[r], bs[r]) <= 1e-10


def test_tuning_cache_file_round_trip(dw, tmp_path, monkeypatch):
    """The autotuner's choices are appended to the tuning file as
    'key T RB pair' lines with block shapes inside the launch limits."""
    import os
    path = os.environ.get("DW_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "dwsolve", "tune.txt")
    dims, kappa = (4, 6, 4, 6), 0.12  # a shape no other test uses
    U = I.gauge_field(dims, "exp", 100, 1, 0.4)
    b = I.gaussian_spinor(dims, 100, 2)
    Ug, bg, x = dw.gauge(dims, kappa, U), dw.spinor(dims, b), dw.spinor(dims)
    dw.cg_solve(Ug, bg, x, dw.params(tol=1e-10, inner="f32"))
    lines = [l.split() for l in open(path).read().splitlines() if "4x6x4x6" in l]
    assert lines
    for key, T, RB, pair in lines:
        T, RB = int(T), int(RB)
        assert T % 32 == 0 and 32 <= T <= 256 and RB >= 1 and T * RB <= 256 and pair in ("0", "1")


def test_solves_from_two_host_threads(dw):
    """Solver calls from two host threads (different systems, precisions and
    lattices, hence different cached plans) are serialised by the library and
    both certify against the oracle."""
    import threading
    import torch
    cases = [((4, 4, 4, 8), 0.12, 101, dict(inner="f16", compress12=1, outer="df64")),
             ((6, 4, 4, 6), 0.118, 102, dict(inner="f32", outer="f64"))]
    fields = []
    for dims, kappa, seed, kw in cases:
        U = I.gauge_field(dims, "exp", seed, 1, 0.4)
        b = I.gaussian_spinor(dims, seed, 2)
        fields.append((dims, kappa, U, b, dw.gauge(dims, kappa, U), dw.spinor(dims, b), dw.spinor(dims),
                       dw.params(tol=1e-10, **kw)))
    torch.cuda.synchronize()
    out, errs = {}, []

    def worker(i):
        try:
            torch.cuda.set_device(0)
            dims, kappa, U, b, Ug, bg, xg, p = fields[i]
            for _ in range(3):
                xg.storage.zero_()
                s, st = dw.cg_solve(Ug, bg, xg, p)
                assert s == dw.DW_OK
            out[i] = xg.download()
        except Exception as e:  # reported below
            errs.append(repr(e))

    th = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for i, (dims, kappa, U, b, *_rest) in enumerate(fields):
        assert _resid(dims, kappa, U, out[i], b) <= 1e-10
