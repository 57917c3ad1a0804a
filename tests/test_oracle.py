"""Pins of the FP64 oracle against facts fixed by the mathematics.

The paper (Sec. 1, Sec. 3.2) poses the problem -- a Dirac-Wilson system solved
by conjugate gradient -- but prints no equation and no worked example, so the
oracle is pinned by:
  * the Clifford algebra of the chosen gamma basis;
  * the free-field (U = 1) momentum-space closed form of D on plane waves,
    with antiperiodic momenta in time;
  * gamma5-hermiticity gamma5 D gamma5 = D^dag and the adjoint identity;
  * gauge covariance under a random SU(3) transformation;
  * dense assembly checked against the matrix-free operator on unit vectors
    and against the closed-form free spectrum, then dense LU solves checked
    against the oracle's CG;
  * the even-odd Schur complement against dense block algebra;
  * the link force against central finite differences.
None of these re-types the stencil formula: each compares the oracle with an
independent statement of the same mathematics.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O
from paper_2001_05218_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def coords(dims):
    V = I.volume(dims)
    s = np.arange(V)
    x = s % dims[0]
    y = (s // dims[0]) % dims[1]
    z = (s // (dims[0] * dims[1])) % dims[2]
    t = s // (dims[0] * dims[1] * dims[2])
    return np.stack([x, y, z, t], axis=1)


def shift(field, dims, mu, step):
    """field(x + step*mu_hat) as a site array (periodic wrap, no sign)."""
    shp = (dims[3], dims[2], dims[1], dims[0]) + field.shape[1:]
    f = field.reshape(shp)
    axis = 3 - mu
    return np.roll(f, -step, axis=axis).reshape(field.shape)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def vdot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


# ------------------------------------------------------------- gamma algebra

def test_clifford_algebra():
    g = [O.gamma(m) for m in range(4)]
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T, atol=0)
        for n in range(4):
            ac = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(ac, 2.0 * (m == n) * np.eye(4), atol=1e-15)
    g5 = O.gamma(4)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)
    for m in range(4):
        assert np.allclose(g5 @ g[m] + g[m] @ g5, 0, atol=1e-15)


# ------------------------------------------------------------- free field

@pytest.mark.parametrize("anti_t", [1, 0])
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 5, 1, 6), (2, 1, 0, 3)])
def test_free_field_plane_wave(anti_t, n):
    dims = (4, 6, 2, 8)
    kappa = 0.137
    V = I.volume(dims)
    U = I.gauge_field(dims, "unit", 0, 0)
    p = np.array([2 * np.pi * n[m] / dims[m] for m in range(4)])
    if anti_t:
        p[3] = (2 * np.pi * n[3] + np.pi) / dims[3]
    rng = np.random.default_rng(7)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    ph = np.exp(1j * coords(dims) @ p)
    psi = ph[:, None, None] * u[None]
    g = [O.gamma(m) for m in range(4)]
    Dp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(g[m] * np.sin(p[m]) for m in range(4))
    expect = ph[:, None, None] * (Dp @ u)[None]
    got = O.dirac(dims, kappa, U, psi, anti_t=anti_t)
    assert rel(got, expect) < 1e-14
    Dpd = Dp.conj().T
    got_d = O.dirac(dims, kappa, U, psi, anti_t=anti_t, dag=True)
    assert rel(got_d, ph[:, None, None] * (Dpd @ u)[None]) < 1e-14


def test_free_field_solve_closed_form():
    """With U = 1 and b a plane wave, x = D(p)^{-1} b exactly."""
    dims = (4, 4, 4, 8)
    kappa = 0.12
    U = I.gauge_field(dims, "unit", 0, 0)
    n = (1, 2, 3, 2)
    p = np.array([2 * np.pi * n[m] / dims[m] for m in range(4)])
    p[3] = (2 * np.pi * n[3] + np.pi) / dims[3]
    u = np.arange(12).reshape(4, 3) + 1j
    ph = np.exp(1j * coords(dims) @ p)
    b = ph[:, None, None] * u[None]
    g = [O.gamma(m) for m in range(4)]
    Dp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(g[m] * np.sin(p[m]) for m in range(4))
    expect = ph[:, None, None] * np.linalg.solve(Dp, u)[None]
    x, it, rr = O.cgnr(dims, kappa, U, b, tol=1e-13)
    assert it > 0 and rr < 1e-13
    assert rel(x, expect) < 1e-12


# ------------------------------------------------------------- symmetries

def _random_setup(dims, seed=11):
    U = I.gauge_field(dims, "haar", seed, 1)
    psi = I.gaussian_spinor(dims, seed, 2)
    eta = I.gaussian_spinor(dims, seed, 3)
    return U, psi, eta


def test_gamma5_hermiticity():
    dims = (4, 2, 6, 4)
    U, psi, _ = _random_setup(dims)
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    lhs = np.einsum("st,vtc->vsc", g5, O.dirac(dims, 0.13, U, np.einsum("st,vtc->vsc", g5, psi)))
    rhs = O.dirac(dims, 0.13, U, psi, dag=True)
    assert rel(lhs, rhs) < 1e-14


def test_adjoint_identity():
    dims = (2, 4, 4, 6)
    U, psi, eta = _random_setup(dims, 5)
    a = vdot(eta, O.dirac(dims, 0.11, U, psi))
    b = vdot(O.dirac(dims, 0.11, U, eta, dag=True), psi)
    assert abs(a - b) / abs(a) < 1e-14


@pytest.mark.parametrize("anti_t", [1, 0])
def test_gauge_covariance(anti_t):
    dims = (4, 4, 2, 6)
    U, psi, _ = _random_setup(dims, 9)
    Om = I.gauge_transform(dims, 9, 7)
    Up = np.empty_like(U)
    for mu in range(4):
        Om_f = shift(Om, dims, mu, +1)
        Up[:, mu] = Om @ U[:, mu] @ np.conj(np.transpose(Om_f, (0, 2, 1)))
    psip = np.einsum("vab,vsb->vsa", Om, psi)
    lhs = O.dirac(dims, 0.12, Up, psip, anti_t=anti_t)
    rhs = np.einsum("vab,vsb->vsa", Om, O.dirac(dims, 0.12, U, psi, anti_t=anti_t))
    assert rel(lhs, rhs) < 1e-14


def test_hop_single_source_support():
    """H applied to a delta source touches only the 8 neighbours, and the
    result there is unitary-equivalent in norm to (1 -/+ gamma) u."""
    dims = (4, 4, 4, 4)
    U, _, _ = _random_setup(dims, 3)
    src = np.zeros((I.volume(dims), 4, 3), dtype=complex)
    y = 1 + 4 * (2 + 4 * (3 + 4 * 0))
    u = np.arange(12).reshape(4, 3) * (1 + 0.5j)
    src[y] = u
    h = O.hop(dims, U, src)
    nz = set(np.nonzero(np.abs(h).sum(axis=(1, 2)) > 0)[0].tolist())
    nb = set()
    for mu in range(4):
        for st in (1, -1):
            idx = np.arange(I.volume(dims)).astype(float)
            nb.add(int(shift(idx, dims, mu, st)[y]))
    assert nz == nb
    g = [O.gamma(m) for m in range(4)]
    for mu in range(4):
        xm = int(shift(np.arange(I.volume(dims)).astype(float), dims, mu, -1)[y])  # y - mu
        xp = int(shift(np.arange(I.volume(dims)).astype(float), dims, mu, +1)[y])  # y + mu
        # norms are invariant under the colour rotation by the link
        assert abs(np.linalg.norm(h[xm]) - np.linalg.norm((np.eye(4) - g[mu]) @ u)) < 1e-12
        assert abs(np.linalg.norm(h[xp]) - np.linalg.norm((np.eye(4) + g[mu]) @ u)) < 1e-12


# ------------------------------------------------------------- dense algebra

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
def test_dense_matches_matrix_free(dims):
    U, _, _ = _random_setup(dims, 21)
    kappa = 0.124
    M = O.dense_dirac(dims, kappa, U)
    N = M.shape[0]
    E = np.eye(N, dtype=complex)
    for j in range(N):
        col = O.dirac(dims, kappa, U, E[j].reshape(-1, 4, 3)).reshape(-1)
        assert np.abs(col - M[:, j]).max() < 1e-14


def test_dense_free_spectrum():
    """Singular values squared of the dense free D are the closed-form
    (1 - 2k sum cos p)^2 + 4 k^2 sum sin^2 p, each 12-fold."""
    dims = (2, 2, 4, 4)
    kappa = 0.13
    U = I.gauge_field(dims, "unit", 0, 0)
    M = O.dense_dirac(dims, kappa, U)
    ev = np.sort(np.linalg.eigvalsh(M.conj().T @ M))
    vals = []
    for nx in range(dims[0]):
        for ny in range(dims[1]):
            for nz in range(dims[2]):
                for nt in range(dims[3]):
                    p = 2 * np.pi * np.array([nx, ny, nz, nt]) / np.array(dims)
                    p[3] += np.pi / dims[3]
                    v = (1 - 2 * kappa * np.cos(p).sum()) ** 2 + 4 * kappa ** 2 * (np.sin(p) ** 2).sum()
                    vals += [v] * 12
    assert np.abs(ev - np.sort(vals)).max() < 1e-13


def test_cgnr_matches_lu():
    dims = (2, 2, 2, 2)
    U, b, _ = _random_setup(dims, 31)
    kappa = 0.12
    M = O.dense_dirac(dims, kappa, U)
    x_lu = sla.lu_solve(sla.lu_factor(M), b.reshape(-1)).reshape(b.shape)
    x, it, rr = O.cgnr(dims, kappa, U, b, tol=1e-13)
    assert it > 0 and rr < 1e-13
    assert rel(x, x_lu) < 1e-11


def test_cg_normal_matches_lu():
    dims = (2, 2, 2, 4)
    U, b, _ = _random_setup(dims, 32)
    kappa = 0.12
    M = O.dense_dirac(dims, kappa, U)
    A = M.conj().T @ M
    x_lu = sla.solve(A, b.reshape(-1), assume_a="her").reshape(b.shape)
    x, it, rr = O.cg_normal(dims, kappa, U, b, tol=1e-13)
    assert it > 0 and rr < 1e-13
    assert rel(x, x_lu) < 1e-10


def _parity(dims):
    return coords(dims).sum(axis=1) % 2


def test_schur_complement_matches_dense_blocks():
    dims = (2, 2, 2, 4)
    U, psi, _ = _random_setup(dims, 41)
    kappa = 0.125
    M = O.dense_dirac(dims, kappa, U)
    par = np.repeat(_parity(dims), 12)
    e, o = np.nonzero(par == 0)[0], np.nonzero(par == 1)[0]
    S = M[np.ix_(e, e)] - M[np.ix_(e, o)] @ np.linalg.solve(M[np.ix_(o, o)], M[np.ix_(o, e)])
    got = O.schur(dims, kappa, U, psi, parity=0).reshape(-1)
    assert np.abs(got[o]).max() == 0
    assert rel(got[e], S @ psi.reshape(-1)[e]) < 1e-14
    # odd-parity Schur complement and the dagger via gamma5
    So = M[np.ix_(o, o)] - M[np.ix_(o, e)] @ np.linalg.solve(M[np.ix_(e, e)], M[np.ix_(e, o)])
    got_o = O.schur(dims, kappa, U, psi, parity=1).reshape(-1)
    assert rel(got_o[o], So @ psi.reshape(-1)[o]) < 1e-14
    got_d = O.schur(dims, kappa, U, psi, parity=0, dag=True).reshape(-1)
    assert rel(got_d[e], S.conj().T @ psi.reshape(-1)[e]) < 1e-14


def test_even_odd_solve_equals_full_solve():
    dims = (2, 2, 4, 4)
    U, b, _ = _random_setup(dims, 43)
    kappa = 0.12
    M = O.dense_dirac(dims, kappa, U)
    x_full = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    be = O.mask_parity(dims, b, 0)
    bo = O.mask_parity(dims, b, 1)
    bhat = be + kappa * O.mask_parity(dims, O.hop(dims, U, bo), 0)
    par = np.repeat(_parity(dims), 12)
    e = np.nonzero(par == 0)[0]
    Sdense = np.zeros((e.size, e.size), dtype=complex)
    for j in range(e.size):
        v = np.zeros(b.size, dtype=complex)
        v[e[j]] = 1
        Sdense[:, j] = O.schur(dims, kappa, U, v.reshape(b.shape), parity=0).reshape(-1)[e]
    xe_vec = np.linalg.solve(Sdense, bhat.reshape(-1)[e])
    xe = np.zeros(b.size, dtype=complex)
    xe[e] = xe_vec
    xe = xe.reshape(b.shape)
    xo = bo + kappa * O.mask_parity(dims, O.hop(dims, U, xe), 1)
    assert rel(xe + xo, x_full) < 1e-12


# ------------------------------------------------------------- force

def _S_dense(dims, kappa, U, phi):
    M = O.dense_dirac(dims, kappa, U)
    A = M.conj().T @ M
    return float(np.real(np.vdot(phi.reshape(-1), np.linalg.solve(A, phi.reshape(-1)))))


def test_force_matches_finite_differences_of_action():
    dims = (2, 2, 2, 4)
    kappa = 0.12
    U, phi, _ = _random_setup(dims, 51)
    M = O.dense_dirac(dims, kappa, U)
    A = M.conj().T @ M
    X = np.linalg.solve(A, phi.reshape(-1)).reshape(phi.shape)
    Y = O.dirac(dims, kappa, U, X)
    G = 2 * O.force(dims, kappa, Y, X)
    h = 1e-5
    rng = np.random.default_rng(3)
    for _ in range(6):
        s, mu, a, c = rng.integers(I.volume(dims)), rng.integers(4), rng.integers(3), rng.integers(3)
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            Up = U.copy(); Up[s, mu, a, c] += h * unit
            Um = U.copy(); Um[s, mu, a, c] -= h * unit
            fd = (_S_dense(dims, kappa, Up, phi) - _S_dense(dims, kappa, Um, phi)) / (2 * h)
            assert abs(fd - part(G[s, mu, a, c])) < 1e-6 * max(1.0, abs(fd))


def _expm_ah(T):
    w, v = np.linalg.eigh(-1j * T)  # -iT is Hermitian
    return (v * np.exp(1j * w)[None, :]) @ v.conj().T


def test_su3_force_matches_group_derivative():
    dims = (2, 2, 2, 4)
    kappa = 0.115
    U, phi, _ = _random_setup(dims, 53)
    M = O.dense_dirac(dims, kappa, U)
    A = M.conj().T @ M
    X = np.linalg.solve(A, phi.reshape(-1)).reshape(phi.shape)
    Y = O.dirac(dims, kappa, U, X)
    G = 2 * O.force(dims, kappa, Y, X)
    P = O.su3_project(G, U)
    # P is traceless anti-Hermitian
    assert np.abs(P + np.conj(np.transpose(P, (0, 1, 3, 2)))).max() < 1e-14
    assert np.abs(np.trace(P, axis1=2, axis2=3)).max() < 1e-14
    rng = np.random.default_rng(4)
    h = 1e-5
    for _ in range(4):
        s, mu = rng.integers(I.volume(dims)), rng.integers(4)
        a = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        T = 0.5 * (a - a.conj().T)
        T -= np.trace(T) / 3 * np.eye(3)
        Up = U.copy(); Up[s, mu] = _expm_ah(h * T) @ U[s, mu]
        Um = U.copy(); Um[s, mu] = _expm_ah(-h * T) @ U[s, mu]
        fd = (_S_dense(dims, kappa, Up, phi) - _S_dense(dims, kappa, Um, phi)) / (2 * h)
        an = np.real(np.trace(P[s, mu].conj().T @ T))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(fd))


def test_source_gradient_finite_differences():
    """L = Re<c, x>, x = (D^dag D)^{-1} b: dL/db = (D^dag D)^{-1} c and
    dL/dU = F(D x, l) + F(D l, x) with l = (D^dag D)^{-1} c."""
    dims = (2, 2, 2, 4)
    kappa = 0.12
    U, b, c = _random_setup(dims, 61)
    M = O.dense_dirac(dims, kappa, U)
    A = M.conj().T @ M

    def L(Uu, bb):
        Mm = O.dense_dirac(dims, kappa, Uu)
        xx = np.linalg.solve(Mm.conj().T @ Mm, bb.reshape(-1))
        return float(np.real(np.vdot(c.reshape(-1), xx)))

    x = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
    lam = np.linalg.solve(A, c.reshape(-1)).reshape(b.shape)
    G = O.force(dims, kappa, O.dirac(dims, kappa, U, x), lam) + O.force(dims, kappa, O.dirac(dims, kappa, U, lam), x)
    h = 1e-5
    rng = np.random.default_rng(5)
    for _ in range(4):
        s, mu, a, cc = rng.integers(I.volume(dims)), rng.integers(4), rng.integers(3), rng.integers(3)
        Up = U.copy(); Up[s, mu, a, cc] += h
        Um = U.copy(); Um[s, mu, a, cc] -= h
        fd = (L(Up, b) - L(Um, b)) / (2 * h)
        assert abs(fd - G[s, mu, a, cc].real) < 1e-6 * max(1.0, abs(fd))
        s2, sp, col = rng.integers(I.volume(dims)), rng.integers(4), rng.integers(3)
        bp = b.copy(); bp[s2, sp, col] += 1j * h
        bm = b.copy(); bm[s2, sp, col] -= 1j * h
        fd = (L(U, bp) - L(U, bm)) / (2 * h)
        assert abs(fd - lam[s2, sp, col].imag) < 1e-6 * max(1.0, abs(fd))


# ---------------------------------------------------------------- second stencil: covariant Laplacian
# M = 1 - kappa K, K = sum_mu [eta U_mu(x) delta_{x+mu} + eta U_mu(x-mu)^dag delta_{x-mu}] on every spin.

@pytest.mark.parametrize("anti_t,n", [(1, (1, 2, 0, 3)), (0, (0, 1, 1, 2)), (1, (2, 0, 1, 0))])
def test_laplace_free_field_plane_wave(anti_t, n):
    """With U = 1 a plane wave is an eigenvector, eigenvalue 1 - 2 kappa sum_mu cos p_mu
    (p_t shifted by pi/L_t when antiperiodic), the same for every spin."""
    dims = (4, 6, 2, 8)
    kappa = 0.12
    U = I.gauge_field(dims, "unit", 0, 0)
    p = np.array([2 * np.pi * n[m] / dims[m] for m in range(4)])
    if anti_t:
        p[3] = (2 * np.pi * n[3] + np.pi) / dims[3]
    rng = np.random.default_rng(5)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    ph = np.exp(1j * coords(dims) @ p)
    psi = ph[:, None, None] * u[None]
    got = O.laplace(dims, kappa, U, psi, anti_t=anti_t)
    assert rel(got, (1 - 2 * kappa * np.cos(p).sum()) * psi) < 1e-14


def test_laplace_is_hermitian_part_of_wilson():
    """(D + D^dag)/2 = 1 - kappa (H + Hdag)/2, and (1 - gamma) + (1 + gamma) = 2:
    the spin-diagonal Laplacian is the Hermitian part of the (independently
    pinned) Wilson operator for the same links and kappa."""
    dims = (4, 2, 4, 6)
    U, psi, _ = _random_setup(dims, 31)
    for anti_t in (1, 0):
        lhs = O.laplace(dims, 0.113, U, psi, anti_t=anti_t)
        rhs = 0.5 * (O.dirac(dims, 0.113, U, psi, anti_t=anti_t) + O.dirac(dims, 0.113, U, psi, anti_t=anti_t, dag=True))
        assert rel(lhs, rhs) < 1e-14


def test_laplace_hermitian_positive_and_gauge_covariant():
    dims = (4, 4, 2, 6)
    U, psi, eta = _random_setup(dims, 33)
    kappa = 0.124
    a = vdot(eta, O.laplace(dims, kappa, U, psi))
    b = vdot(O.laplace(dims, kappa, U, eta), psi)
    assert abs(a - b) / abs(a) < 1e-14
    q = vdot(psi, O.laplace(dims, kappa, U, psi))
    assert abs(q.imag) < 1e-12 * abs(q) and q.real > (1 - 8 * kappa) * vdot(psi, psi).real * (1 - 1e-12)
    Om = I.gauge_transform(dims, 33, 7)
    Up = np.empty_like(U)
    for mu in range(4):
        Up[:, mu] = Om @ U[:, mu] @ np.conj(np.transpose(shift(Om, dims, mu, +1), (0, 2, 1)))
    lhs = O.laplace(dims, kappa, Up, np.einsum("vab,vsb->vsa", Om, psi))
    rhs = np.einsum("vab,vsb->vsa", Om, O.laplace(dims, kappa, U, psi))
    assert rel(lhs, rhs) < 1e-14


def test_laplace_cg_matches_dense_solve():
    """Plain CG on M against an LU solve of the dense Hermitian part of the
    dense Wilson matrix (on a lattice small enough to assemble)."""
    dims = (2, 2, 2, 4)
    U, psi, _ = _random_setup(dims, 35)
    kappa = 0.121
    Dd = O.dense_dirac(dims, kappa, U)
    M = 0.5 * (Dd + Dd.conj().T)
    x_lu = np.linalg.solve(M, psi.reshape(-1))
    x, it, rr = O.cg_laplace(dims, kappa, U, psi, tol=1e-13)
    assert it > 0 and rr < 1e-12
    assert rel(x.reshape(-1), x_lu) < 1e-11
