"""Python binding of libdw.so (include/dw.h): argument marshalling only.

Every function of the C ABI is exposed under its own name and returns the
dw_status; `check(status)` turns a non-zero status into DwError carrying
dw_last_error().  The Field class gives a handle whose device memory comes
from PyTorch (a uint8 CUDA tensor) wrapped through dw_field_wrap, so
PyTorch's caching allocator owns it; streams are PyTorch's current CUDA
stream.  Nothing here computes: all work runs in the library's kernels, and
there is no fallback -- if libdw.so is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdw.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libdw.so is not built (run paper_2001_05218_gb300/build.py or __graft_entry__.build()); "
                      "there is no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)

# ------------------------------------------------------------------ enums
DW_OK, DW_ERR_ARG, DW_ERR_SHAPE, DW_ERR_PRECISION, DW_ERR_OOM, DW_ERR_CUDA, \
    DW_ERR_NOT_CONVERGED, DW_ERR_BREAKDOWN, DW_ERR_TIMEOUT = range(9)
STATUS_NAMES = ["DW_OK", "DW_ERR_ARG", "DW_ERR_SHAPE", "DW_ERR_PRECISION", "DW_ERR_OOM", "DW_ERR_CUDA",
                "DW_ERR_NOT_CONVERGED", "DW_ERR_BREAKDOWN", "DW_ERR_TIMEOUT"]
DW_F64, DW_F32, DW_F16, DW_BF16, DW_DF64, DW_I16 = range(6)
DW_GAUGE, DW_SPINOR_FULL, DW_SPINOR_EVEN, DW_SPINOR_ODD = range(4)
PREC = {"f64": DW_F64, "f32": DW_F32, "f16": DW_F16, "bf16": DW_BF16, "df64": DW_DF64, "i16": DW_I16}


class dw_lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("t_antiperiodic", ctypes.c_int), ("kappa", ctypes.c_double)]


class dw_solver_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("inner", ctypes.c_int),
                ("delta", ctypes.c_double), ("eo", ctypes.c_int), ("compress12", ctypes.c_int),
                ("recompute_fwd", ctypes.c_int), ("tile", ctypes.c_int), ("check_every", ctypes.c_int),
                ("timeout_s", ctypes.c_double), ("verify_normal", ctypes.c_int), ("outer", ctypes.c_int),
                ("defect_correction", ctypes.c_int)]


class dw_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 64), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class dw_solver_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("true_rel_resid", ctypes.c_double),
                ("normal_rel_resid", ctypes.c_double), ("time_ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I = ctypes.c_int
_LP = ctypes.POINTER(dw_lattice)
_FP = ctypes.c_void_p  # dw_field*
_SIGS = {
    "dw_field_bytes": [_LP, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)],
    "dw_field_alloc": [_LP, _I, _I, _I, _I, ctypes.POINTER(_FP)],
    "dw_field_wrap": [_LP, _I, _I, _I, _I, _P, ctypes.c_size_t, ctypes.POINTER(_FP)],
    "dw_field_free": [_FP],
    "dw_field_upload": [_FP, _P, _P],
    "dw_field_download": [_FP, _P, _P],
    "dw_field_import": [_FP, _P, _P],
    "dw_field_export": [_FP, _P, _P],
    "dw_field_info": [_FP, _LP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "dw_apply": [_FP, _FP, _FP, _P],
    "dw_apply_dag": [_FP, _FP, _FP, _P],
    "dw_normal_apply": [_FP, _FP, _FP, _P],
    "dw_apply_norm": [_FP, _FP, _FP, _I, ctypes.POINTER(ctypes.c_double), _P],
    "dw_field_mark_modified": [_FP],
    "dw_apply_noalloc": [_FP, _FP, _FP, _I, _P],
    "dw_solver_params_default": [ctypes.POINTER(dw_solver_params)],
    "dw_cg_solve": [_FP, _FP, _FP, ctypes.POINTER(dw_solver_params), ctypes.POINTER(dw_solver_stats), _P],
    "dw_cg_solve_batched": [_I, ctypes.POINTER(_FP), ctypes.POINTER(_FP), ctypes.POINTER(_FP),
                            ctypes.POINTER(dw_solver_params), ctypes.POINTER(dw_solver_stats), _P],
    "dw_cg_solve_normal": [_FP, _FP, _FP, ctypes.POINTER(dw_solver_params), ctypes.POINTER(dw_solver_stats), _P],
    "dw_cg_solve_laplace": [_FP, _FP, _FP, ctypes.POINTER(dw_solver_params), ctypes.POINTER(dw_solver_stats), _P],
    "dw_laplace_apply": [_FP, _FP, _FP, _P],
    "dw_profile_start": [_I],
    "dw_profile_stop": [ctypes.POINTER(dw_profile_entry), _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_longlong)],
    "dw_cg_backward": [_FP, _FP, _FP, _FP, _FP, _FP, _I, ctypes.POINTER(dw_solver_params),
                       ctypes.POINTER(dw_solver_stats), _P],
}
for _name, _args in _SIGS.items():
    if hasattr(_lib, _name):
        _f = getattr(_lib, _name)
        _f.argtypes = _args
        _f.restype = ctypes.c_int
        globals()[_name] = _f
_lib.dw_last_error.restype = ctypes.c_char_p
_lib.dw_last_error.argtypes = []
_lib.dw_version.restype = ctypes.c_char_p
_lib.dw_version.argtypes = []


def dw_last_error() -> str:
    return _lib.dw_last_error().decode()


def dw_version() -> str:
    return _lib.dw_version().decode()


class DwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 9 else status, msg))
        self.status = status


def check(status: int) -> int:
    if status != DW_OK:
        raise DwError(status, dw_last_error())
    return status


def symbols():
    """Names exported by the loaded library (for the ABI test)."""
    return sorted(n for n in list(_SIGS) + ["dw_last_error", "dw_version"] if hasattr(_lib, n))


# ------------------------------------------------------------------ helpers over torch
def _torch():
    import torch
    return torch


def current_stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def lattice(dims, kappa=0.0, t_antiperiodic=1) -> dw_lattice:
    lat = dw_lattice()
    for i in range(4):
        lat.dims[i] = int(dims[i])
    lat.t_antiperiodic = int(t_antiperiodic)
    lat.kappa = float(kappa)
    return lat


def params(**kw) -> dw_solver_params:
    p = dw_solver_params()
    check(dw_solver_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k in ("inner", "outer") and isinstance(v, str):
            v = PREC[v]
        setattr(p, k, v)
    return p


class Field:
    """A field whose device memory is a zero-filled PyTorch uint8 CUDA tensor."""

    def __init__(self, lat: dw_lattice, kind: int, prec: int = DW_F64, compress12: int = 0, nrhs: int = 1,
                 device=None):
        torch = _torch()
        self.lat, self.kind, self.prec, self.compress12, self.nrhs = lat, kind, prec, compress12, nrhs
        nb = ctypes.c_size_t(0)
        check(dw_field_bytes(ctypes.byref(lat), kind, prec, compress12, nrhs, ctypes.byref(nb)))
        self.nbytes = nb.value
        # 256-byte aligned: allocate a little extra and offset
        self.storage = torch.zeros(self.nbytes + 256, dtype=torch.uint8, device=device or "cuda")
        base = self.storage.data_ptr()
        self.offset = (-base) % 256
        self.ptr = base + self.offset
        h = _FP()
        check(dw_field_wrap(ctypes.byref(lat), kind, prec, compress12, nrhs, ctypes.c_void_p(self.ptr),
                            ctypes.c_size_t(self.nbytes), ctypes.byref(h)))
        self.handle = h

    # canonical complex128 shapes
    def canonical_shape(self):
        V = int(np.prod(list(self.lat.dims)))
        if self.kind == DW_GAUGE:
            return (V, 4, 3, 3)
        n = V if self.kind == DW_SPINOR_FULL else V // 2
        return (self.nrhs, n, 4, 3) if self.nrhs > 1 else (n, 4, 3)

    def upload(self, host: np.ndarray, stream=None):
        a = np.ascontiguousarray(host, dtype=np.complex128)
        assert a.size == int(np.prod(self.canonical_shape())), (a.shape, self.canonical_shape())
        # pageable source: the copy is staged before the call returns
        check(dw_field_upload(self.handle, ctypes.c_void_p(a.ctypes.data), stream or current_stream()))
        return self

    def download(self, stream=None) -> np.ndarray:
        out = np.empty(self.canonical_shape(), dtype=np.complex128)
        check(dw_field_download(self.handle, ctypes.c_void_p(out.ctypes.data), stream or current_stream()))
        _torch().cuda.current_stream().synchronize()
        return out

    def import_(self, t, stream=None):
        """From a CUDA complex128 tensor in canonical order."""
        torch = _torch()
        assert t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()
        check(dw_field_import(self.handle, ctypes.c_void_p(t.data_ptr()), stream or current_stream()))
        return self

    def export(self, stream=None):
        torch = _torch()
        t = torch.empty(self.canonical_shape(), dtype=torch.complex128, device=self.storage.device)
        check(dw_field_export(self.handle, ctypes.c_void_p(t.data_ptr()), stream or current_stream()))
        return t

    def mark_modified(self):
        """Declare that self.storage was written in place (dw_field_mark_modified)."""
        check(dw_field_mark_modified(self.handle))
        return self

    def free(self):
        if getattr(self, "handle", None):
            dw_field_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def gauge(dims, kappa, U, prec=DW_F64, compress12=0, t_antiperiodic=1):
    lat = lattice(dims, kappa, t_antiperiodic)
    f = Field(lat, DW_GAUGE, prec, compress12)
    f.upload(U.reshape(-1, 4, 3, 3))
    return f


def spinor(dims, psi=None, kind=DW_SPINOR_FULL, prec=DW_F64, nrhs=1, kappa=0.0, t_antiperiodic=1):
    lat = lattice(dims, kappa, t_antiperiodic)
    f = Field(lat, kind, prec, 0, nrhs)
    if psi is not None:
        f.upload(psi)
    return f


def apply(U: Field, x: Field, out: Field, dag=False, normal=False):
    fn = dw_normal_apply if normal else (dw_apply_dag if dag else dw_apply)
    check(fn(U.handle, x.handle, out.handle, current_stream()))
    return out


def apply_norm(U: Field, x: Field, out: Field, dag=False):
    """out = D x (or D^dag x); returns |out_r|^2 per right-hand side from the
    library's FP64 grid reduction (dw_apply_norm)."""
    n = (ctypes.c_double * x.nrhs)()
    check(dw_apply_norm(U.handle, x.handle, out.handle, 1 if dag else 0, n, current_stream()))
    return np.array(n[:], dtype=np.float64)


def cg_solve(U: Field, b: Field, x: Field, p: dw_solver_params = None, raise_on_fail=True):
    p = p or params()
    st = (dw_solver_stats * b.nrhs)()
    s = dw_cg_solve(U.handle, b.handle, x.handle, ctypes.byref(p), st, current_stream())
    if raise_on_fail:
        check(s)
    return s, [st[i].as_dict() for i in range(b.nrhs)]


def cg_solve_normal(U: Field, b: Field, x: Field, p: dw_solver_params = None, raise_on_fail=True):
    p = p or params()
    st = (dw_solver_stats * b.nrhs)()
    s = dw_cg_solve_normal(U.handle, b.handle, x.handle, ctypes.byref(p), st, current_stream())
    if raise_on_fail:
        check(s)
    return s, [st[i].as_dict() for i in range(b.nrhs)]


def laplace_apply(U: Field, x: Field, out: Field):
    """out = M x for the covariant Laplacian M = 1 - kappa K (Schur complement on parity fields)."""
    check(dw_laplace_apply(U.handle, x.handle, out.handle, current_stream()))
    return out


def cg_solve_laplace(U: Field, b: Field, x: Field, p: dw_solver_params = None, raise_on_fail=True):
    """M x = b for the covariant Laplacian by plain CG (see dw_cg_solve_laplace)."""
    p = p or params()
    st = (dw_solver_stats * b.nrhs)()
    s = dw_cg_solve_laplace(U.handle, b.handle, x.handle, ctypes.byref(p), st, current_stream())
    if raise_on_fail:
        check(s)
    return s, [st[i].as_dict() for i in range(b.nrhs)]


def cg_solve_batched(Us, bs, xs, p: dw_solver_params = None, raise_on_fail=True):
    p = p or params()
    n = len(Us)
    arr = lambda fs: (_FP * n)(*[f.handle.value for f in fs])  # noqa: E731
    nr = bs[0].nrhs
    st = (dw_solver_stats * (n * nr))()
    s = dw_cg_solve_batched(n, arr(Us), arr(bs), arr(xs), ctypes.byref(p), st, current_stream())
    if raise_on_fail:
        check(s)
    return s, [st[i].as_dict() for i in range(n * nr)]


def profile_start(time_stencils=False):
    check(dw_profile_start(1 if time_stencils else 0))


def profile_stop():
    """Returns ({name: {launches, total_ms, bytes, flops}}, total kernel launches)."""
    ents = (dw_profile_entry * 32)()
    n = ctypes.c_int(0)
    nl = ctypes.c_longlong(0)
    check(dw_profile_stop(ents, 32, ctypes.byref(n), ctypes.byref(nl)))
    out = {}
    for i in range(min(n.value, 32)):
        e = ents[i]
        out[e.name.decode()] = dict(launches=e.launches, total_ms=e.total_ms, bytes=e.bytes, flops=e.flops)
    return out, nl.value
