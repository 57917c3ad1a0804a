"""GPU operator parity: dw_apply / dw_apply_dag / dw_normal_apply through the
C ABI against the FP64 oracle on the same seeded inputs.

Bars: FP64 storage <= 1e-13 and FP32 <= 1e-6 per-site relative norm; the
double-float format (FP64-sized storage, ~49-bit arithmetic on the FP32
pipes) is held to the FP64 bar;
16-bit storage (FP16 / BF16 operands, spin projection rounded to 16 bits, FP32
accumulation) is held to bounds derived from the unit roundoff of the storage
type (2^-11 for FP16 values scaled to [-1, 1] per site, 2^-8 for BF16) times
the few roundings on the path; 16-bit fixed point (I16) to 2e-4 (half a unit
of 1/32767 of the site maximum on input, links and output, FP32 arithmetic).
Lattices are chosen so that half volumes span several thread blocks and end
in a partial block (192, 960 and 1620 sites per parity with 128-site blocks).
"""
import numpy as np
import pytest

from helpers import parity_of_sites, site_err
from oracle import oracle as O
from paper_2001_05218_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "df64": 1e-13, "f32": 1e-6, "f16": 4e-3, "bf16": 3e-2, "i16": 2e-4}
DIMS = [(4, 4, 4, 6), (8, 6, 4, 10), (6, 10, 6, 6)]


@pytest.fixture(scope="module")
def dw():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_05218_gb300 import dw as m
    return m


def _setup(dims, seed=101, kind="haar"):
    U = I.gauge_field(dims, kind, seed, 1, 0.5)
    psi = I.gaussian_spinor(dims, seed, 2)
    return U, psi


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("anti_t", [1, 0])
def test_apply_full_f64(dw, dims, anti_t):
    kappa = 0.1234
    U, psi = _setup(dims)
    Ug = dw.gauge(dims, kappa, U, t_antiperiodic=anti_t)
    x = dw.spinor(dims, psi)
    out = dw.spinor(dims)
    for dag in (False, True):
        dw.apply(Ug, x, out, dag=dag)
        ref = O.dirac(dims, kappa, U, psi, anti_t=anti_t, dag=dag)
        assert site_err(out.download(), ref) <= TOL["f64"]


@pytest.mark.parametrize("dims", DIMS[:2])
@pytest.mark.parametrize("prec,c12", [("f64", 0), ("f64", 1), ("df64", 0), ("df64", 1), ("f32", 0), ("f32", 1),
                                      ("f16", 0), ("f16", 1), ("bf16", 0), ("bf16", 1), ("i16", 0), ("i16", 1)])
def test_apply_precisions(dw, dims, prec, c12):
    kappa = 0.118
    U, psi = _setup(dims, 7)
    P = dw.PREC[prec]
    Ug = dw.gauge(dims, kappa, U, prec=P, compress12=c12)
    x = dw.spinor(dims, psi, prec=P)
    out = dw.spinor(dims, prec=P)
    for dag in (False, True):
        dw.apply(Ug, x, out, dag=dag)
        ref = O.dirac(dims, kappa, U, psi, dag=dag)
        e = site_err(out.download(), ref)
        assert e <= TOL[prec], (prec, c12, dag, e)


SCHUR_CASES = [("f64", 0), ("df64", 0), ("f32", 0), ("f32", 1), ("i16", 0), ("i16", 1),
               ("f16", 0), ("f16", 1), ("bf16", 0), ("bf16", 1)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("prec,c12", SCHUR_CASES)
def test_apply_schur(dw, dims, parity, prec, c12):
    """The even-odd Schur complement Dhat = 1 - kappa^2 H_pq H_qp, its adjoint
    and Dhat^dag Dhat, site by site against the oracle, in every storage
    precision with 18- and 12-real links: the 16-bit 12-real operator is the
    one the mixed-precision solver iterates with."""
    kappa = 0.125
    U, psi = _setup(dims, 17)
    par = parity_of_sites(dims)
    P = dw.PREC[prec]
    kind = dw.DW_SPINOR_EVEN if parity == 0 else dw.DW_SPINOR_ODD
    Ug = dw.gauge(dims, kappa, U, prec=P, compress12=c12)
    sub = psi[par == parity]
    x = dw.spinor(dims, sub, kind=kind, prec=P)
    out = dw.spinor(dims, kind=kind, prec=P)
    full = np.zeros_like(psi)
    full[par == parity] = sub
    for dag in (False, True):
        dw.apply(Ug, x, out, dag=dag)
        ref = O.schur(dims, kappa, U, full, parity=parity, dag=dag)[par == parity]
        e = site_err(out.download(), ref)
        assert e <= TOL[prec], (prec, c12, dag, e)
    dw.apply(Ug, x, out, normal=True)
    t = O.schur(dims, kappa, U, full, parity=parity)
    ref = O.schur(dims, kappa, U, t, parity=parity, dag=True)[par == parity]
    assert site_err(out.download(), ref) <= 10 * TOL[prec]


NORM_CASES = [("f16", 1, "even"), ("f16", 1, "odd"), ("f16", 0, "even"), ("bf16", 1, "even"), ("bf16", 0, "odd"),
              ("i16", 1, "even"), ("f32", 1, "even"), ("f32", 0, "full"), ("f16", 1, "full"), ("f64", 0, "even"),
              ("f64", 0, "full"), ("df64", 0, "even")]


@pytest.mark.parametrize("dims", DIMS[1:])
@pytest.mark.parametrize("prec,c12,kind", NORM_CASES)
def test_apply_norm_reducing_epilogue(dw, dims, prec, c12, kind):
    """dw_apply_norm runs the solver's reducing epilogue (out = x + c H t with
    |out|^2 reduced in FP64 over the grid): its output must match the oracle
    site by site, and the returned |out|^2 must match |oracle|^2 to the
    storage precision's bound (the norm is of the value before its rounding
    to storage, so it carries the operator's error, not the store's)."""
    kappa = 0.121
    U, psi = _setup(dims, 19)
    par = parity_of_sites(dims)
    P = dw.PREC[prec]
    k = {"even": dw.DW_SPINOR_EVEN, "odd": dw.DW_SPINOR_ODD, "full": dw.DW_SPINOR_FULL}[kind]
    Ug = dw.gauge(dims, kappa, U, prec=P, compress12=c12)
    if kind == "full":
        full, keep = psi, np.ones(len(psi), dtype=bool)
    else:
        pty = 0 if kind == "even" else 1
        keep = par == pty
        full = np.where(keep[:, None, None], psi, 0)
    x = dw.spinor(dims, full[keep], kind=k, prec=P)
    out = dw.spinor(dims, kind=k, prec=P)
    for dag in (False, True):
        n2 = dw.apply_norm(Ug, x, out, dag=dag)
        if kind == "full":
            ref = O.dirac(dims, kappa, U, psi, dag=dag)
        else:
            ref = O.schur(dims, kappa, U, full, parity=pty, dag=dag)[keep]
        e = site_err(out.download(), ref)
        assert e <= TOL[prec], (prec, c12, kind, dag, e)
        ref2 = float(np.vdot(ref.reshape(-1), ref.reshape(-1)).real)
        assert abs(n2[0] - ref2) <= 2 * TOL[prec] * ref2, (n2[0], ref2)


def test_apply_norm_multi_rhs_and_repeatability(dw):
    """Per right-hand side norms of a 12-RHS FP16 field, and bitwise-equal
    norms on repeated calls (fixed-order reduction)."""
    dims, kappa, n = (8, 6, 4, 10), 0.12, 12
    U, _ = _setup(dims, 41)
    par = parity_of_sites(dims)
    psis = np.stack([I.gaussian_spinor(dims, 41, 10 + r)[par == 0] * (1 + r) for r in range(n)])
    Ug = dw.gauge(dims, kappa, U, prec=dw.DW_F16, compress12=1)
    x = dw.spinor(dims, psis, kind=dw.DW_SPINOR_EVEN, prec=dw.DW_F16, nrhs=n)
    out = dw.spinor(dims, kind=dw.DW_SPINOR_EVEN, prec=dw.DW_F16, nrhs=n)
    a = dw.apply_norm(Ug, x, out)
    b = dw.apply_norm(Ug, x, out)
    assert np.array_equal(a, b)
    got = out.download()
    for r in range(n):
        full = np.zeros((int(np.prod(dims)), 4, 3), dtype=np.complex128)
        full[par == 0] = psis[r]
        ref = O.schur(dims, kappa, U, full, parity=0)[par == 0]
        assert site_err(got[r], ref) <= TOL["f16"]
        ref2 = float(np.vdot(ref.reshape(-1), ref.reshape(-1)).real)
        assert abs(a[r] - ref2) <= 2 * TOL["f16"] * ref2


def test_normal_apply_full(dw):
    dims, kappa = (4, 4, 4, 6), 0.11
    U, psi = _setup(dims, 23)
    Ug = dw.gauge(dims, kappa, U)
    x = dw.spinor(dims, psi)
    out = dw.spinor(dims)
    dw.apply(Ug, x, out, normal=True)
    assert site_err(out.download(), O.normal(dims, kappa, U, psi)) <= 1e-13


def test_multi_rhs_apply(dw):
    dims, kappa, n = (8, 6, 4, 10), 0.12, 5
    U, _ = _setup(dims, 29)
    psis = np.stack([I.gaussian_spinor(dims, 29, 10 + r) for r in range(n)])
    Ug = dw.gauge(dims, kappa, U, prec=dw.DW_F32)
    x = dw.spinor(dims, psis, prec=dw.DW_F32, nrhs=n)
    out = dw.spinor(dims, prec=dw.DW_F32, nrhs=n)
    dw.apply(Ug, x, out)
    got = out.download()
    for r in range(n):
        assert site_err(got[r], O.dirac(dims, kappa, U, psis[r])) <= TOL["f32"]


@pytest.mark.parametrize("prec,c12", [("f16", 1), ("bf16", 1), ("f16", 0), ("i16", 1), ("f32", 1)])
@pytest.mark.parametrize("kind", ["full", "even"])
def test_multi_rhs_apply_12_sources(dw, prec, c12, kind):
    """12 right-hand sides (the spin-colour sources of the multi-RHS solve) in
    16-bit and FP32 storage with 12-real links: every column against the
    oracle, full lattice and even-site Schur complement, both D and D^dag."""
    dims, kappa, n = (6, 10, 6, 6), 0.12, 12
    U, _ = _setup(dims, 43)
    par = parity_of_sites(dims)
    P = dw.PREC[prec]
    psis = np.stack([I.gaussian_spinor(dims, 43, 10 + r) for r in range(n)])
    if kind == "even":
        psis = np.where((par == 0)[None, :, None, None], psis, 0)
        x = dw.spinor(dims, psis[:, par == 0], kind=dw.DW_SPINOR_EVEN, prec=P, nrhs=n)
        out = dw.spinor(dims, kind=dw.DW_SPINOR_EVEN, prec=P, nrhs=n)
    else:
        x = dw.spinor(dims, psis, prec=P, nrhs=n)
        out = dw.spinor(dims, prec=P, nrhs=n)
    Ug = dw.gauge(dims, kappa, U, prec=P, compress12=c12)
    for dag in (False, True):
        dw.apply(Ug, x, out, dag=dag)
        got = out.download()
        for r in range(n):
            if kind == "even":
                ref = O.schur(dims, kappa, U, psis[r], parity=0, dag=dag)[par == 0]
            else:
                ref = O.dirac(dims, kappa, U, psis[r], dag=dag)
            e = site_err(got[r], ref)
            assert e <= TOL[prec], (prec, c12, kind, dag, r, e)


def test_layout_roundtrip_is_exact(dw):
    dims = (6, 10, 6, 6)
    U, psi = _setup(dims, 31)
    par = parity_of_sites(dims)
    assert np.array_equal(dw.spinor(dims, psi).download(), psi)
    assert np.array_equal(dw.spinor(dims, psi[par == 1], kind=dw.DW_SPINOR_ODD).download(), psi[par == 1])
    g = dw.gauge(dims, 0.1, U)
    lat = g.lat
    assert np.array_equal(g.download(), U)
    g12 = dw.gauge(dims, 0.1, U, compress12=1)
    assert np.abs(g12.download() - U).max() < 1e-14  # row 2 rebuilt from SU(3) unitarity


def test_golden_fixture_on_gpu(dw):
    import os
    from test_golden_and_inputs import load_golden
    meta, Dpsi, Ddag, _ = load_golden()
    dims, kappa, seed = meta["dims"], meta["kappa"], meta["seed"]
    U = I.gauge_field(dims, "haar", seed, 1)
    psi = I.gaussian_spinor(dims, seed, 2)
    Ug = dw.gauge(dims, kappa, U)
    x = dw.spinor(dims, psi)
    out = dw.spinor(dims)
    dw.apply(Ug, x, out)
    assert site_err(out.download(), Dpsi) <= 1e-13
    dw.apply(Ug, x, out, dag=True)
    assert site_err(out.download(), Ddag) <= 1e-13


def test_apply_rejects_mismatches(dw):
    dims = (4, 4, 4, 6)
    U, psi = _setup(dims)
    Ug = dw.gauge(dims, 0.1, U)
    x = dw.spinor(dims, psi)
    y32 = dw.spinor(dims, prec=dw.DW_F32)
    assert dw.dw_apply(Ug.handle, x.handle, y32.handle, dw.current_stream()) == dw.DW_ERR_SHAPE or \
        dw.dw_apply(Ug.handle, x.handle, y32.handle, dw.current_stream()) == dw.DW_ERR_PRECISION
    other = dw.spinor((4, 4, 4, 8))
    assert dw.dw_apply(Ug.handle, x.handle, other.handle, dw.current_stream()) == dw.DW_ERR_SHAPE
    assert dw.dw_apply(Ug.handle, x.handle, x.handle, dw.current_stream()) == dw.DW_ERR_ARG


def test_pinned_host_roundtrip_is_exact(dw):
    """Pinned host buffers are read and written directly by the layout kernels."""
    import ctypes
    import torch
    dims = (8, 6, 4, 10)
    U, psi = _setup(dims, 37)
    hp = torch.from_numpy(psi.reshape(-1).view(np.float64).copy()).pin_memory()
    hU = torch.from_numpy(U.reshape(-1).view(np.float64).copy()).pin_memory()
    x = dw.spinor(dims)
    g = dw.Field(dw.lattice(dims, 0.1), dw.DW_GAUGE)
    dw.check(dw.dw_field_upload(x.handle, ctypes.c_void_p(hp.data_ptr()), dw.current_stream()))
    dw.check(dw.dw_field_upload(g.handle, ctypes.c_void_p(hU.data_ptr()), dw.current_stream()))
    out = torch.zeros_like(hp).pin_memory()
    dw.check(dw.dw_field_download(x.handle, ctypes.c_void_p(out.data_ptr()), dw.current_stream()))
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy().view(np.complex128).reshape(psi.shape), psi)
    assert np.array_equal(x.download(), psi)
    assert np.array_equal(g.download(), U)


def test_double_float_conversion_accuracy(dw):
    """binary64 -> (hi, lo) float pair -> binary64 through a DW_DF64 field:
    relative error <= 2^-47 for magnitudes 1e-20 .. 1e20, zeros exact."""
    dims = (4, 4, 4, 4)
    rng = np.random.default_rng(5)
    mag = 10.0 ** rng.uniform(-20, 20, size=(256, 4, 3))
    psi = (rng.normal(size=(256, 4, 3)) + 1j * rng.normal(size=(256, 4, 3))) * mag
    psi[0] = 0.0
    psi[1, 0, 0] = -1.0 + 0.5j
    f = dw.spinor(dims, psi, prec=dw.DW_DF64)
    back = f.download()
    assert np.all(back[0] == 0)
    rel = np.abs(back - psi) / np.maximum(np.abs(psi), 1e-300)
    assert rel[1:].max() <= 2.0 ** -47

