"""Boundary behaviour of field handles over caller-owned memory: a gauge
field wrapped around a tensor that the caller rewrites in place must be
re-derived (dw_field_mark_modified) so that the mixed-precision solver's
inner (FP16) and outer (double-float) link copies follow the new links."""
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


@pytest.mark.parametrize("inner,c12,outer", [("f16", 1, "df64"), ("f32", 0, "f64")])
def test_wrapped_gauge_rewritten_in_place(dw, inner, c12, outer):
    dims, kappa = (8, 8, 8, 8), 0.12
    U1 = I.gauge_field(dims, "exp", 81, 1, 0.5)
    U2 = I.gauge_field(dims, "exp", 82, 1, 0.5)
    b = I.gaussian_spinor(dims, 81, 2)
    p = dw.params(tol=1e-10, inner=inner, compress12=c12, outer=outer)
    Ug = dw.gauge(dims, kappa, U1)
    bg = dw.spinor(dims, b)
    x1 = dw.spinor(dims)
    s, _ = dw.cg_solve(Ug, bg, x1, p)  # builds the derived link copies of U1
    assert s == dw.DW_OK
    assert _resid(dims, kappa, U1, x1.download(), b) <= 1e-10
    # the caller rewrites the wrapped memory itself (bytes of a field holding U2)
    other = dw.gauge(dims, kappa, U2)
    Ug.storage[Ug.offset:Ug.offset + Ug.nbytes].copy_(other.storage[other.offset:other.offset + other.nbytes])
    Ug.mark_modified()
    x2 = dw.spinor(dims)
    s, st = dw.cg_solve(Ug, bg, x2, p)
    assert s == dw.DW_OK and st[0]["true_rel_resid"] <= 1e-10
    assert _resid(dims, kappa, U2, x2.download(), b) <= 1e-10


def test_mark_modified_rejects_null(dw):
    assert dw.dw_field_mark_modified(None) == dw.DW_ERR_ARG
