"""Host transfers through dw_field_upload / dw_field_download at sizes that
take the chunked path (64 MiB and more: DMA copies on the library's copy
stream, layout kernels on the caller's stream).

Checks: exact round trips with chunk boundaries inside a right-hand side and
inside the lattice; ordering against work already queued on the caller's
stream and against work queued after the call; derived link copies refreshed
chunk by chunk by an upload (the solve that follows equals, bit for bit, one
on a fresh field).
"""
import ctypes

import numpy as np
import pytest

from paper_2001_05218_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DIMS = (16, 16, 16, 32)  # V = 131072: links 75.5 MB (2 chunks), 4-rhs spinor 100.7 MB (3 chunks)


@pytest.fixture(scope="module")
def dw():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_05218_gb300 import dw as m
    return m


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).view(np.float64).copy()).pin_memory()


def _up(dw, f, h):
    dw.check(dw.dw_field_upload(f.handle, ctypes.c_void_p(h.data_ptr()), dw.current_stream()))


def _down(dw, f, h):
    dw.check(dw.dw_field_download(f.handle, ctypes.c_void_p(h.data_ptr()), dw.current_stream()))


@pytest.mark.parametrize("kind,nrhs", [("full", 4), ("odd", 8)])
def test_chunked_spinor_roundtrip_is_exact(dw, kind, nrhs):
    import torch
    V = int(np.prod(DIMS))
    n = V if kind == "full" else V // 2
    rng = np.random.default_rng(nrhs)
    psi = rng.normal(size=(nrhs, n, 4, 3)) + 1j * rng.normal(size=(nrhs, n, 4, 3))
    assert psi.nbytes >= 64 << 20
    k = dw.DW_SPINOR_FULL if kind == "full" else dw.DW_SPINOR_ODD
    f = dw.Field(dw.lattice(DIMS), k, dw.DW_F64, 0, nrhs)
    h = _pinned(psi)
    _up(dw, f, h)
    out = torch.zeros_like(h).pin_memory()
    _down(dw, f, out)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(out.numpy().view(np.complex128).reshape(psi.shape), psi)
    # FP32 storage: the round trip is the binary32 rounding of each component
    f32 = dw.Field(dw.lattice(DIMS), k, dw.DW_F32, 0, nrhs)
    _up(dw, f32, h)
    _down(dw, f32, out)
    torch.cuda.current_stream().synchronize()
    want = psi.real.astype(np.float32).astype(np.float64) + 1j * psi.imag.astype(np.float32).astype(np.float64)
    assert np.array_equal(out.numpy().view(np.complex128).reshape(psi.shape), want)


def test_chunked_gauge_roundtrip_is_exact(dw):
    import torch
    U = I.gauge_field(DIMS, "exp", 3, 1, 0.6).reshape(-1, 4, 3, 3)
    assert U.nbytes >= 64 << 20
    g = dw.Field(dw.lattice(DIMS, 0.1), dw.DW_GAUGE)
    h = _pinned(U)
    _up(dw, g, h)
    out = torch.zeros_like(h).pin_memory()
    _down(dw, g, out)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(out.numpy().view(np.complex128).reshape(U.shape), U)


def test_chunked_transfers_keep_stream_order(dw):
    """An upload reads a pinned buffer that a copy queued just before it on the
    same stream is still writing; work queued after a download reads the
    buffer that the download's copies write."""
    import torch
    V = int(np.prod(DIMS))
    gen = torch.Generator(device="cuda").manual_seed(11)
    src = torch.randn(4 * V * 24, dtype=torch.float64, device="cuda", generator=gen)
    h = torch.empty(src.numel(), dtype=torch.float64).pin_memory()
    f = dw.Field(dw.lattice(DIMS), dw.DW_SPINOR_FULL, dw.DW_F64, 0, 4)
    for _ in range(3):
        src.mul_(-1.0)
        h.copy_(src, non_blocking=True)  # queued on the current stream, not waited for
        _up(dw, f, h)
        back = torch.empty_like(h).pin_memory()
        _down(dw, f, back)
        dev = back.to("cuda", non_blocking=True)  # queued after the download
        torch.cuda.current_stream().synchronize()
        assert torch.equal(dev, src)


def test_upload_refreshes_derived_links(dw):
    """A gauge field that already holds FP16 and double-float copies of its
    links gets new links by a chunked upload: the mixed solve that follows is
    bit for bit the one on a freshly made field."""
    import torch
    kappa = 0.12
    U1 = I.gauge_field(DIMS, "exp", 5, 1, 0.6).reshape(-1, 4, 3, 3)
    U2 = I.gauge_field(DIMS, "exp", 6, 1, 0.6).reshape(-1, 4, 3, 3)
    b = I.gaussian_spinor(DIMS, 7, 2)
    p = dw.params(tol=1e-10, inner="f16", outer="df64", compress12=1)
    A = dw.Field(dw.lattice(DIMS, kappa), dw.DW_GAUGE)
    _up(dw, A, _pinned(U1))
    bf = dw.spinor(DIMS, b, kappa=kappa)
    xa = dw.spinor(DIMS, kappa=kappa)
    dw.cg_solve(A, bf, xa, p)  # makes the derived copies of U1
    _up(dw, A, _pinned(U2))
    xa = dw.spinor(DIMS, kappa=kappa)
    _, sa = dw.cg_solve(A, bf, xa, p)
    B = dw.Field(dw.lattice(DIMS, kappa), dw.DW_GAUGE)
    _up(dw, B, _pinned(U2))
    xb = dw.spinor(DIMS, kappa=kappa)
    _, sb = dw.cg_solve(B, bf, xb, p)
    torch.cuda.synchronize()
    assert sa[0]["iters"] == sb[0]["iters"]
    assert np.array_equal(xa.download(), xb.download())


def test_transfers_under_stream_capture(dw):
    """Captured into a CUDA graph (one copy and one kernel per call while the
    stream is capturing), an upload and a download replay exactly."""
    import torch
    V = int(np.prod(DIMS))
    rng = np.random.default_rng(21)
    psi = rng.normal(size=(4, V, 4, 3)) + 1j * rng.normal(size=(4, V, 4, 3))
    f = dw.Field(dw.lattice(DIMS), dw.DW_SPINOR_FULL, dw.DW_F64, 0, 4)
    h = _pinned(psi)
    out = torch.zeros_like(h).pin_memory()
    _up(dw, f, h)  # the library's pool and copy stream exist before capture
    _down(dw, f, out)
    torch.cuda.synchronize()
    f.storage.zero_()
    out.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        dw.check(dw.dw_field_upload(f.handle, ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
        dw.check(dw.dw_field_download(f.handle, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
    torch.cuda.synchronize()
    assert not out.any()  # nothing ran during capture
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy().view(np.complex128).reshape(psi.shape), psi)


def test_import_refreshes_derived_links(dw):
    """dw_field_import (device canonical array) into a gauge field that holds
    derived link copies: the next solve equals, bit for bit, one on a fresh
    field."""
    import torch
    dims, kappa = (8, 8, 8, 16), 0.12
    U1 = I.gauge_field(dims, "exp", 15, 1, 0.5).reshape(-1, 4, 3, 3)
    U2 = I.gauge_field(dims, "exp", 16, 1, 0.5).reshape(-1, 4, 3, 3)
    b = I.gaussian_spinor(dims, 17, 2)
    p = dw.params(tol=1e-10, inner="f16", compress12=1, outer="df64")
    A = dw.gauge(dims, kappa, U1)
    bf = dw.spinor(dims, b, kappa=kappa)
    xa = dw.spinor(dims, kappa=kappa)
    dw.cg_solve(A, bf, xa, p)  # derived copies of U1
    A.import_(torch.from_numpy(U2).to("cuda"))
    xa = dw.spinor(dims, kappa=kappa)
    _, sa = dw.cg_solve(A, bf, xa, p)
    B = dw.gauge(dims, kappa, U2)
    xb = dw.spinor(dims, kappa=kappa)
    _, sb = dw.cg_solve(B, bf, xb, p)
    torch.cuda.synchronize()
    assert sa[0]["iters"] == sb[0]["iters"]
    assert np.array_equal(xa.download(), xb.download())
