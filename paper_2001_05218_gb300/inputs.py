"""Seeded synthetic inputs for the Wilson-Dirac solver (gauge links, sources).

This module is shared by the tests, the oracle checks and the benchmark.  It
holds no part of the method's arithmetic (no Dirac operator, no solver): it
only draws random numbers and shapes them into fields in the canonical host
layout

    spinor  psi[site, spin, colour]            complex128, shape (V, 4, 3)
    gauge   U[site, mu, row, col]              complex128, shape (V, 4, 3, 3)
    site  = x + Lx*(y + Ly*(z + Lz*t)),  mu = 0..3 = x, y, z, t.

Random numbers come from a counter-based generator: output i of stream k of
seed s is splitmix64 (Steele, Lea & Flood 2014) applied to a per-stream key
plus i times the golden-ratio increment, so any slice of any field can be
regenerated independently.  Uniforms use the top 53 bits, Gaussians use the
Box-Muller transform.  The draw order is site-major, then mu, then row, col,
then (re, im).

Link ensembles (the paper uses the 3x3 complex link matrices U of its Fig. 1
but gives no ensemble; these are synthetic stand-ins):
  * Haar SU(3): QR of a complex Gaussian matrix with the phases of R's
    diagonal moved into Q (Mezzadri 2007), then Q * det(Q)^(-1/3) on the
    principal branch so det = 1.
  * exp(i a H): H a random traceless Hermitian matrix, U = exp(i a H) formed
    from the eigen-decomposition of H.  Small a gives near-unit, smooth links.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 200105218


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        a = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN], dtype=np.uint64))
        b = _mix(np.array([np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + a[0]], dtype=np.uint64))
    return b[0]


def uint64_stream(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the counter-based splitmix64 stream."""
    key = _key(seed, stream)
    with np.errstate(over="ignore"):
        i = np.arange(start, start + count, dtype=np.uint64) + np.uint64(1)
        return _mix(key + i * _GOLDEN)


def uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in (0, 1)."""
    u = uint64_stream(seed, stream, start, count)
    return ((u >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def gaussian(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Standard normal doubles; pairs (2j, 2j+1) come from one Box-Muller draw."""
    assert start % 2 == 0 and count % 2 == 0
    u = uniform(seed, stream, start, count).reshape(-1, 2)
    rad = np.sqrt(-2.0 * np.log(u[:, 0]))
    ang = 2.0 * np.pi * u[:, 1]
    out = np.empty((u.shape[0], 2))
    out[:, 0] = rad * np.cos(ang)
    out[:, 1] = rad * np.sin(ang)
    return out.reshape(-1)


def complex_gaussian(seed: int, stream: int, start: int, count: int, var: float = 1.0) -> np.ndarray:
    """count complex numbers with E|z|^2 = var (re, im independent)."""
    g = gaussian(seed, stream, 2 * start, 2 * count).reshape(-1, 2)
    s = np.sqrt(var / 2.0)
    return (g[:, 0] + 1j * g[:, 1]) * s


def volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


# ---------------------------------------------------------------- sources

def gaussian_spinor(dims, seed: int, stream: int) -> np.ndarray:
    """Spinor with re and im of every component i.i.d. N(0, 1)."""
    V = volume(dims)
    z = complex_gaussian(seed, stream, 0, V * 12, var=2.0)
    return z.reshape(V, 4, 3)


def point_source(dims, spin: int, colour: int, site: int = 0) -> np.ndarray:
    psi = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    psi[site, spin, colour] = 1.0
    return psi


# ---------------------------------------------------------------- links

_CHUNK = 1 << 18  # matrices per generation chunk (bounds host memory)


def _gaussian_matrices(seed, stream, first, n):
    z = complex_gaussian(seed, stream, first * 9, n * 9, var=1.0)
    return z.reshape(n, 3, 3)


def haar_su3(n: int, seed: int, stream: int, first: int = 0) -> np.ndarray:
    """n Haar-distributed SU(3) matrices (matrix index first .. first+n-1)."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for c0 in range(0, n, _CHUNK):
        m = min(_CHUNK, n - c0)
        a = _gaussian_matrices(seed, stream, first + c0, m)
        q, r = np.linalg.qr(a)
        d = np.diagonal(r, axis1=1, axis2=2)
        ph = d / np.abs(d)
        q = q * ph[:, None, :]
        det = np.linalg.det(q)
        q = q * (det ** (-1.0 / 3.0))[:, None, None]
        out[c0:c0 + m] = q
    return out


def exp_su3(n: int, amplitude: float, seed: int, stream: int, first: int = 0) -> np.ndarray:
    """n matrices exp(i a H), H random traceless Hermitian (A + A^dag)/2 minus
    its trace part, A complex Gaussian with E|A_ij|^2 = 1."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    eye = np.eye(3)
    for c0 in range(0, n, _CHUNK):
        m = min(_CHUNK, n - c0)
        a = _gaussian_matrices(seed, stream, first + c0, m)
        h = 0.5 * (a + np.conj(np.transpose(a, (0, 2, 1))))
        tr = np.trace(h, axis1=1, axis2=2).real
        h = h - (tr / 3.0)[:, None, None] * eye
        w, v = np.linalg.eigh(h)
        ph = np.exp(1j * amplitude * w)
        out[c0:c0 + m] = (v * ph[:, None, :]) @ np.conj(np.transpose(v, (0, 2, 1)))
    return out


def gauge_field(dims, kind: str, seed: int, stream: int, amplitude: float = 0.0) -> np.ndarray:
    """Gauge field U[V, 4, 3, 3]; kind 'haar', 'exp' or 'unit'."""
    V = volume(dims)
    if kind == "unit":
        u = np.broadcast_to(np.eye(3, dtype=np.complex128), (V * 4, 3, 3)).copy()
    elif kind == "haar":
        u = haar_su3(V * 4, seed, stream)
    elif kind == "exp":
        u = exp_su3(V * 4, amplitude, seed, stream)
    else:
        raise ValueError(kind)
    return u.reshape(V, 4, 3, 3)


def gauge_transform(dims, seed: int, stream: int) -> np.ndarray:
    """Random SU(3) matrix per site, Omega[V, 3, 3] (Haar)."""
    return haar_su3(volume(dims), seed, stream)


# ---------------------------------------------------------------- workloads

# Synthetic workloads.  kappa and link ensembles follow the benchmark
# definitions of this project (the paper states none of them).
WORKLOADS = {
    "wilson_4x4x4x4_haar": dict(dims=(4, 4, 4, 4), kappa=0.12, links="haar", amplitude=0.0, index=0),
    "wilson_16x16x16x32_exp0.4": dict(dims=(16, 16, 16, 32), kappa=0.124, links="exp", amplitude=0.4, index=1),
    "wilson_32x32x32x64_exp0.6": dict(dims=(32, 32, 32, 64), kappa=0.1245, links="exp", amplitude=0.6, index=2),
    "wilson_24x24x24x48_exp0.4_12src": dict(dims=(24, 24, 24, 48), kappa=None, links="exp", amplitude=0.4, index=3),
    "wilson_16x16x16x32_exp0.4_grad": dict(dims=(16, 16, 16, 32), kappa=0.12, links="exp", amplitude=0.4, index=4),
    # profiling size: stencil traffic above the 129 MB L2, ~1.5 GB on the device
    "wilson_32x32x32x32_exp0.6": dict(dims=(32, 32, 32, 32), kappa=0.1245, links="exp", amplitude=0.6, index=5),
}

RAGGED_DIMS = [(8, 8, 8, 8), (8, 8, 8, 16), (12, 12, 12, 24), (16, 16, 16, 16),
               (16, 16, 16, 32), (16, 16, 16, 32), (12, 12, 12, 12), (20, 20, 20, 40)]

STREAM_LINKS, STREAM_SOURCE, STREAM_SOURCE2, STREAM_KAPPA, STREAM_OMEGA = 1, 2, 3, 4, 5


def workload_seed(index: int) -> int:
    return BASE_SEED + index


def make_workload(name: str, with_source: bool = True):
    """Returns (dims, kappa, U, b) for one named single-lattice workload."""
    w = WORKLOADS[name]
    seed = workload_seed(w["index"])
    dims = w["dims"]
    kappa = w["kappa"]
    if kappa is None:
        kappa = 0.115 + 0.010 * float(uniform(seed, STREAM_KAPPA, 0, 1)[0])
    U = gauge_field(dims, w["links"], seed, STREAM_LINKS, w["amplitude"])
    b = gaussian_spinor(dims, seed, STREAM_SOURCE) if with_source else None
    return dims, kappa, U, b


def ragged_batch(seed_index: int = 3):
    """The 8 independent lattices of the ragged batch: list of (dims, kappa, U, b)."""
    seed = workload_seed(seed_index)
    kap = 0.115 + 0.010 * uniform(seed, STREAM_KAPPA, 2, len(RAGGED_DIMS))
    out = []
    for i, dims in enumerate(RAGGED_DIMS):
        s = seed * 1000 + 17 * (i + 1)
        U = gauge_field(dims, "exp", s, STREAM_LINKS, 0.4)
        b = gaussian_spinor(dims, s, STREAM_SOURCE)
        out.append((dims, float(kap[i]), U, b))
    return out
