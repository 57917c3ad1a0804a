"""The solver's two execution paths: the CUDA graph of the CG loop and the
host-stepped loop that runs while the launch profiler times stencils
(dw_profile_start(1)).  They launch the same kernels in the same order, so
every mode must give bitwise the same solution and iteration count, and the
profiler must report the stencil categories it timed."""
import numpy as np
import pytest

from paper_2001_05218_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DIMS, KAPPA = (8, 8, 8, 16), 0.12


@pytest.fixture(scope="module")
def dw():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_05218_gb300 import dw as m
    return m


CASES = [
    ("wilson", dict(inner="f16", compress12=1, outer="df64")),
    ("wilson", dict(inner="f32", outer="f64")),
    ("wilson", dict(inner="f16", compress12=1, outer="df64", eo=0)),
    ("wilson", dict(inner="bf16", outer="df64", nrhs=3)),
    ("normal", dict(inner="f32", outer="df64")),
    ("laplace", dict(inner="f16", compress12=1, outer="df64")),
]


@pytest.mark.parametrize("op,kw", CASES)
def test_graph_and_stepped_loops_agree(dw, op, kw):
    import torch
    kw = dict(kw)
    nrhs = kw.pop("nrhs", 1)
    U = I.gauge_field(DIMS, "exp", 31, 1, 0.5)
    b = np.stack([I.gaussian_spinor(DIMS, 32, 2 + r) for r in range(nrhs)]) if nrhs > 1 else \
        I.gaussian_spinor(DIMS, 32, 2)
    kappa = 0.11 if op == "laplace" else KAPPA
    Ug = dw.gauge(DIMS, kappa, U)
    bg = dw.spinor(DIMS, b, nrhs=nrhs, kappa=kappa)
    p = dw.params(tol=1e-10, maxiter=5000, **kw)
    solve = {"wilson": dw.cg_solve, "normal": dw.cg_solve_normal, "laplace": dw.cg_solve_laplace}[op]
    out = []
    for stepped in (False, True):
        xg = dw.spinor(DIMS, nrhs=nrhs, kappa=kappa)
        if stepped:
            dw.profile_start(time_stencils=True)
        s, st = solve(Ug, bg, xg, p)
        prof = dw.profile_stop()[0] if stepped else None
        torch.cuda.synchronize()
        out.append((xg.download(), [x["iters"] for x in st], [x["true_rel_resid"] for x in st], prof))
    (x0, it0, r0, _), (x1, it1, r1, prof) = out
    assert it0 == it1
    assert max(r0) <= 1e-10
    assert np.array_equal(x0, x1)
    assert prof and any(k.startswith("hop ") or k.startswith("laplace ") for k in prof)
    assert all(v["launches"] > 0 and v["total_ms"] > 0 for v in prof.values())
