"""Golden regression fixture of the oracle and checks of the seeded inputs."""
import os

import numpy as np

from oracle import oracle as O
from paper_2001_05218_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dirac_2x2x2x4.txt")


def load_golden():
    meta = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("# dims"):
                tok = line[2:].split()
                meta["dims"] = tuple(int(v) for v in tok[1:5])
                meta["kappa"] = float(tok[6])
                meta["seed"] = int(tok[8])
    rows = np.loadtxt(GOLDEN)
    V = I.volume(meta["dims"])
    cols = rows[:, 3:].reshape(V, 4, 3, 6)
    Dpsi = cols[..., 0] + 1j * cols[..., 1]
    Ddag = cols[..., 2] + 1j * cols[..., 3]
    x = cols[..., 4] + 1j * cols[..., 5]
    return meta, Dpsi, Ddag, x


def test_oracle_reproduces_golden():
    meta, Dpsi, Ddag, x = load_golden()
    dims, kappa, seed = meta["dims"], meta["kappa"], meta["seed"]
    U = I.gauge_field(dims, "haar", seed, 1)
    psi = I.gaussian_spinor(dims, seed, 2)
    assert np.abs(O.dirac(dims, kappa, U, psi) - Dpsi).max() < 1e-13
    assert np.abs(O.dirac(dims, kappa, U, psi, dag=True) - Ddag).max() < 1e-13
    # the stored solution satisfies D x = psi
    assert np.linalg.norm(O.dirac(dims, kappa, U, x) - psi) / np.linalg.norm(psi) < 1e-13


def test_haar_links_are_su3():
    u = I.haar_su3(2000, 1, 1)
    eye = np.eye(3)
    assert np.abs(np.conj(np.transpose(u, (0, 2, 1))) @ u - eye).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-14
    # Haar: E|U_ij|^2 = 1/3, E U_ij = 0
    assert abs(np.mean(np.abs(u) ** 2) - 1 / 3) < 0.01
    assert np.abs(u.mean(axis=0)).max() < 0.05


def test_exp_links_are_su3_and_near_unit():
    u = I.exp_su3(2000, 0.4, 2, 1)
    eye = np.eye(3)
    assert np.abs(np.conj(np.transpose(u, (0, 2, 1))) @ u - eye).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-14
    tr = np.trace(u, axis1=1, axis2=2).real.mean() / 3
    assert 0.7 < tr < 1.0
    u0 = I.exp_su3(10, 0.0, 2, 1)
    assert np.abs(u0 - eye).max() < 1e-15


def test_generator_is_counter_based_and_gaussian():
    a = I.gaussian(7, 3, 0, 4000)
    b = I.gaussian(7, 3, 1000, 2000)
    assert np.array_equal(a[1000:3000], b)
    g = I.gaussian(99, 1, 0, 400000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
    assert not np.array_equal(I.gaussian(7, 4, 0, 10), a[:10])
    psi = I.gaussian_spinor((8, 8, 8, 8), 5, 2)
    assert psi.shape == (4096, 4, 3)
    assert abs(np.mean(psi.real ** 2) - 1) < 0.05 and abs(np.mean(psi.imag ** 2) - 1) < 0.05


GOLDEN_LAPLACE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "laplace_2x2x2x4.txt")


def load_golden_laplace():
    meta = {}
    with open(GOLDEN_LAPLACE) as f:
        for line in f:
            if line.startswith("# dims"):
                tok = line[2:].split()
                meta["dims"] = tuple(int(v) for v in tok[1:5])
                meta["kappa"] = float(tok[6])
                meta["seed"] = int(tok[8])
    rows = np.loadtxt(GOLDEN_LAPLACE)
    V = I.volume(meta["dims"])
    cols = rows[:, 3:].reshape(V, 4, 3, 4)
    return meta, cols[..., 0] + 1j * cols[..., 1], cols[..., 2] + 1j * cols[..., 3]


def test_oracle_reproduces_laplace_golden():
    meta, Mpsi, x = load_golden_laplace()
    dims, kappa, seed = meta["dims"], meta["kappa"], meta["seed"]
    U = I.gauge_field(dims, "haar", seed, 1)
    psi = I.gaussian_spinor(dims, seed, 2)
    assert np.abs(O.laplace(dims, kappa, U, psi) - Mpsi).max() < 1e-13
    assert np.linalg.norm(O.laplace(dims, kappa, U, x) - psi) / np.linalg.norm(psi) < 1e-13
