"""dw_apply_noalloc: the operator application for callers that must not
allocate GPU memory when they call (GPU memory already held by another
framework's caching allocator, latency-critical loops where an allocation
would synchronise the device, fixed memory budgets).  Its result must match
dw_apply's on two calls in a row -- the fixed scratch array keeps the previous
call's contents, which must not leak into the next result -- and fields too
large for the array must be refused with a clear error."""
import numpy as np
import pytest

from helpers import parity_of_sites, site_err
from paper_2001_05218_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "df64": 1e-13, "f16": 1e-6, "bf16": 1e-6, "i16": 1e-6}  # same kernels as dw_apply
# against the FP64 oracle: the per-site bounds of the operator parity tests
TOL_ORACLE = {"f64": 1e-13, "df64": 1e-13, "f32": 1e-6, "f16": 4e-3, "bf16": 3e-2, "i16": 2e-4}


@pytest.fixture(scope="module")
def dw():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_05218_gb300 import dw as m
    return m


@pytest.mark.parametrize("prec,c12", [("f64", 0), ("f32", 0), ("df64", 0), ("f16", 0), ("i16", 0),
                                      ("bf16", 0), ("f16", 1), ("bf16", 1), ("f32", 1)])
@pytest.mark.parametrize("dagger", [0, 1])
def test_noalloc_matches_dw_apply_on_two_calls(dw, prec, c12, dagger):
    from oracle import oracle as O
    dims, kappa = (8, 6, 4, 10), 0.1234
    P = dw.PREC[prec]
    U = I.gauge_field(dims, "exp", 71, 1, 0.5)
    par = parity_of_sites(dims)
    Ug = dw.gauge(dims, kappa, U, prec=P, compress12=c12)
    outs = []
    for call in range(2):  # two different sources in a row through the same scratch
        psi_full = I.gaussian_spinor(dims, 71, 10 + call)
        psi = psi_full[par == 0]
        x = dw.spinor(dims, psi, kind=dw.DW_SPINOR_EVEN, prec=P)
        ref = dw.spinor(dims, kind=dw.DW_SPINOR_EVEN, prec=P)
        got = dw.spinor(dims, kind=dw.DW_SPINOR_EVEN, prec=P)
        dw.apply(Ug, x, ref, dag=bool(dagger))
        dw.check(dw.dw_apply_noalloc(Ug.handle, x.handle, got.handle, dagger, dw.current_stream()))
        g, r = got.download(), ref.download()
        assert site_err(g, r) <= TOL[prec]
        full = np.where((par == 0)[:, None, None], psi_full, 0)
        oref = O.schur(dims, kappa, U, full, parity=0, dag=bool(dagger))[par == 0]
        assert site_err(g, oref) <= TOL_ORACLE[prec]
        outs.append(g)
    assert not np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_noalloc_full_lattice(dw, prec):
    """Full-lattice fields take no scratch: D on all sites in one launch."""
    from oracle import oracle as O
    dims, kappa = (6, 10, 6, 6), 0.12
    P = dw.PREC[prec]
    U = I.gauge_field(dims, "haar", 73, 1)
    psi = I.gaussian_spinor(dims, 73, 2)
    Ug = dw.gauge(dims, kappa, U, prec=P, compress12=1 if prec == "f16" else 0)
    x = dw.spinor(dims, psi, prec=P)
    got = dw.spinor(dims, prec=P)
    for dagger in (0, 1):
        dw.check(dw.dw_apply_noalloc(Ug.handle, x.handle, got.handle, dagger, dw.current_stream()))
        assert site_err(got.download(), O.dirac(dims, kappa, U, psi, dag=bool(dagger))) <= TOL_ORACLE[prec]


def test_noalloc_multi_rhs_odd_parity(dw):
    dims, kappa, n = (4, 4, 4, 6), 0.12, 3
    U = I.gauge_field(dims, "haar", 72, 1)
    par = parity_of_sites(dims)
    psis = np.stack([I.gaussian_spinor(dims, 72, 20 + r)[par == 1] for r in range(n)])
    Ug = dw.gauge(dims, kappa, U)
    x = dw.spinor(dims, psis, kind=dw.DW_SPINOR_ODD, nrhs=n)
    ref = dw.spinor(dims, kind=dw.DW_SPINOR_ODD, nrhs=n)
    got = dw.spinor(dims, kind=dw.DW_SPINOR_ODD, nrhs=n)
    for _ in range(2):
        dw.apply(Ug, x, ref)
        dw.check(dw.dw_apply_noalloc(Ug.handle, x.handle, got.handle, 0, dw.current_stream()))
        assert site_err(got.download(), ref.download()) <= TOL["f64"]


def test_noalloc_refuses_fields_beyond_its_array(dw):
    dims = (32, 32, 32, 32)  # FP64 even field: 524288 sites * 192 B = 96 MiB > 32 MiB
    lat = dw.lattice(dims, 0.12)
    Ug = dw.Field(lat, dw.DW_GAUGE, dw.DW_F64)
    x = dw.Field(lat, dw.DW_SPINOR_EVEN, dw.DW_F64)
    y = dw.Field(lat, dw.DW_SPINOR_EVEN, dw.DW_F64)
    s = dw.dw_apply_noalloc(Ug.handle, x.handle, y.handle, 0, dw.current_stream())
    assert s == dw.DW_ERR_SHAPE
    assert "scratch" in dw.dw_last_error()
