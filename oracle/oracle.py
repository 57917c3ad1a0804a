"""ctypes front end of the FP64 oracle (dw_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package's smoke check
and by the benchmark's CPU-baseline leg -- never by the product library.
Arrays are numpy complex128 in the canonical host layout
(psi[V, 4, 3], U[V, 4, 3, 3], site = x + Lx*(y + Ly*(z + Lz*t))).

Which passage each function follows is stated in dw_oracle.c; this file
only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_dw.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile dw_oracle.c into liboracle_dw.so (gcc, OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        for name, args, res in [
            ("or_gamma", [I, P], None),
            ("or_hop", [P, I, P, P, P], None),
            ("or_hop_dag", [P, I, P, P, P], None),
            ("or_dirac", [P, I, D, P, P, P], None),
            ("or_dirac_dag", [P, I, D, P, P, P], None),
            ("or_normal", [P, I, D, P, P, P], None),
            ("or_mask_parity", [P, P, I], None),
            ("or_schur", [P, I, D, P, P, P, I, I], None),
            ("or_cgnr", [P, I, D, P, P, P, D, I, P], I),
            ("or_cg_normal", [P, I, D, P, P, P, D, I, P], I),
            ("or_laplace", [P, I, D, P, P, P], None),
            ("or_cg_laplace", [P, I, D, P, P, P, D, I, P], I),
            ("or_dense_dirac", [P, I, D, P, P], None),
            ("or_force", [P, I, D, P, P, P], None),
            ("or_su3_project", [ctypes.c_long, P, P, P], None),
            ("or_num_threads", [], I),
            ("or_set_num_threads", [I], None),
        ]:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(v) for v in dims])


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.ctypes.data


def gamma(mu: int) -> np.ndarray:
    """gamma_mu for mu = 0..3 (x, y, z, t); mu = 4 gives gamma_5."""
    g = np.zeros((4, 4), dtype=np.complex128)
    lib().or_gamma(mu, g.ctypes.data)
    return g


def _volume(dims):
    return int(np.prod(dims))


def hop(dims, U, psi, anti_t=1, dag=False):
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    (lib().or_hop_dag if dag else lib().or_hop)(_dims(dims), anti_t, pu, pp, out.ctypes.data)
    return out


def dirac(dims, kappa, U, psi, anti_t=1, dag=False):
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    (lib().or_dirac_dag if dag else lib().or_dirac)(_dims(dims), anti_t, kappa, pu, pp, out.ctypes.data)
    return out


def normal(dims, kappa, U, psi, anti_t=1):
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    lib().or_normal(_dims(dims), anti_t, kappa, pu, pp, out.ctypes.data)
    return out


def mask_parity(dims, psi, keep):
    out = np.array(psi, dtype=np.complex128, copy=True)
    lib().or_mask_parity(_dims(dims), out.ctypes.data, keep)
    return out


def schur(dims, kappa, U, psi, parity=0, anti_t=1, dag=False):
    """Schur complement on `parity`; full-lattice arrays in and out."""
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    lib().or_schur(_dims(dims), anti_t, kappa, pu, pp, out.ctypes.data, parity, 1 if dag else 0)
    return out


def cgnr(dims, kappa, U, b, tol=1e-12, maxiter=100000, anti_t=1, x0=None):
    """x with D x = b by CG on the normal equations; returns (x, iters, rel_resid)."""
    U, pu = _c(U)
    b, pb = _c(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    rr = ctypes.c_double(0)
    it = lib().or_cgnr(_dims(dims), anti_t, kappa, pu, pb, x.ctypes.data, tol, maxiter, ctypes.byref(rr))
    return x, it, rr.value


def cg_normal(dims, kappa, U, b, tol=1e-12, maxiter=100000, anti_t=1):
    """x = (D^dag D)^{-1} b by plain CG; returns (x, iters, rel_resid)."""
    U, pu = _c(U)
    b, pb = _c(b)
    x = np.zeros_like(b)
    rr = ctypes.c_double(0)
    it = lib().or_cg_normal(_dims(dims), anti_t, kappa, pu, pb, x.ctypes.data, tol, maxiter, ctypes.byref(rr))
    return x, it, rr.value


def laplace(dims, kappa, U, psi, anti_t=1):
    """Gauge-covariant Laplacian in hopping form, psi - kappa * K psi (spin-diagonal)."""
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    lib().or_laplace(_dims(dims), anti_t, kappa, pu, pp, out.ctypes.data)
    return out


def cg_laplace(dims, kappa, U, b, tol=1e-12, maxiter=100000, anti_t=1):
    """x = M^{-1} b for the Laplacian M by plain CG; returns (x, iters, rel_resid)."""
    U, pu = _c(U)
    b, pb = _c(b)
    x = np.zeros_like(b)
    rr = ctypes.c_double(0)
    it = lib().or_cg_laplace(_dims(dims), anti_t, kappa, pu, pb, x.ctypes.data, tol, maxiter, ctypes.byref(rr))
    return x, it, rr.value


def dense_dirac(dims, kappa, U, anti_t=1):
    U, pu = _c(U)
    N = 12 * _volume(dims)
    M = np.empty((N, N), dtype=np.complex128)
    lib().or_dense_dirac(_dims(dims), anti_t, kappa, pu, M.ctypes.data)
    return M


def force(dims, kappa, Y, X, anti_t=1):
    """F(Y, X)[V, 4, 3, 3]: -Re<Y, dD X> = Re sum tr(F^dag dU)."""
    Y, py = _c(Y)
    X, px = _c(X)
    F = np.empty((_volume(dims), 4, 3, 3), dtype=np.complex128)
    lib().or_force(_dims(dims), anti_t, kappa, py, px, F.ctypes.data)
    return F


def su3_project(G, U):
    G, pg = _c(G)
    U, pu = _c(U)
    P = np.empty_like(G)
    lib().or_su3_project(G.size // 9, pg, pu, P.ctypes.data)
    return P


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> None:
    """Thread count of the oracle's OpenMP loops."""
    lib().or_set_num_threads(int(n))
