"""GPU differentiation: dw_cg_backward and the autograd.Function front ends,
checked against the oracle's link force (itself pinned to finite
differences), against FP64 central finite differences of GPU solves on 4^4
and 8^4 lattices, and by torch.autograd.gradcheck on a 2^4 lattice."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2001_05218_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_05218_gb300 import autograd as AG
    from paper_2001_05218_gb300 import dw
    return torch, dw, AG


def _tight(dw, inner="f64"):
    return dw.params(tol=1e-13, inner=inner, maxiter=100000)


def _backward(dw, dims, kappa, U, phi, grad_x=None, su3=0, p=None):
    Ug = dw.gauge(dims, kappa, U)
    pg = dw.spinor(dims, phi)
    gx = dw.spinor(dims, grad_x) if grad_x is not None else None
    gb = dw.spinor(dims)
    gU = dw.Field(Ug.lat, dw.DW_GAUGE)
    st = (dw.dw_solver_stats * 2)()
    dw.check(dw.dw_cg_backward(Ug.handle, pg.handle, gx.handle if gx else None, None, gb.handle, gU.handle, su3,
                               ctypes.byref(p or _tight(dw)), st, dw.current_stream()))
    return gb.download(), gU.download(), st


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 4, 4, 6)])
def test_action_force_matches_oracle(env, dims):
    torch, dw, _ = env
    kappa = 0.12
    U = I.gauge_field(dims, "exp", 61, 1, 0.4)
    phi = I.gaussian_spinor(dims, 61, 2)
    gphi, G, st = _backward(dw, dims, kappa, U, phi)
    X, it, rr = O.cg_normal(dims, kappa, U, phi, tol=1e-14)
    Gref = 2 * O.force(dims, kappa, O.dirac(dims, kappa, U, X), X)
    assert _rel(gphi, 2 * X) < 1e-10
    assert _rel(G, Gref) < 1e-10
    _, P, _ = _backward(dw, dims, kappa, U, phi, su3=1)
    assert _rel(P, O.su3_project(Gref, U)) < 1e-10


def test_source_mode_gradients_match_oracle(env):
    torch, dw, _ = env
    dims, kappa = (4, 4, 4, 4), 0.118
    U = I.gauge_field(dims, "exp", 62, 1, 0.4)
    b = I.gaussian_spinor(dims, 62, 2)
    g = I.gaussian_spinor(dims, 62, 3)
    gb, G, st = _backward(dw, dims, kappa, U, b, grad_x=g)
    x, _, _ = O.cg_normal(dims, kappa, U, b, tol=1e-14)
    lam, _, _ = O.cg_normal(dims, kappa, U, g, tol=1e-14)
    Gref = O.force(dims, kappa, O.dirac(dims, kappa, U, x), lam) + O.force(dims, kappa, O.dirac(dims, kappa, U, lam), x)
    assert _rel(gb, lam) < 1e-10
    assert _rel(G, Gref) < 1e-10


def _expm_ah(T):
    w, v = np.linalg.eigh(-1j * T)
    return (v * np.exp(1j * w)[None, :]) @ v.conj().T


@pytest.mark.parametrize("dims,inner", [((4, 4, 4, 4), "f64"), ((8, 8, 8, 8), "f64"), ((4, 4, 4, 4), "f32"),
                                        ((4, 4, 4, 4), "f16")])
def test_su3_force_finite_differences(env, dims, inner):
    """dS/deps along U -> exp(eps T) U at a few links, FP64 central differences
    of GPU solves, against Re tr(P^dag T) from the GPU su(3) force (the force
    itself from a mixed-precision adjoint when inner = f32 or f16)."""
    torch, dw, _ = env
    kappa = 0.12
    U = I.gauge_field(dims, "exp", 63, 1, 0.4)
    phi = I.gaussian_spinor(dims, 63, 2)
    _, P, _ = _backward(dw, dims, kappa, U, phi, su3=1, p=dw.params(tol=1e-10, inner=inner, maxiter=100000))
    Ug = dw.gauge(dims, kappa, U)
    pg = dw.spinor(dims, phi)

    def S(Uh):
        Ug.upload(Uh)
        x = dw.spinor(dims)
        dw.cg_solve_normal(Ug, pg, x, _tight(dw))
        return float(np.real(np.vdot(phi.reshape(-1), x.download().reshape(-1))))

    rng = np.random.default_rng(7)
    h = 1e-4
    for _ in range(3):
        s, mu = rng.integers(I.volume(dims)), rng.integers(4)
        a = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        T = 0.5 * (a - a.conj().T)
        T -= np.trace(T) / 3 * np.eye(3)
        Up = U.copy(); Up[s, mu] = _expm_ah(h * T) @ U[s, mu]
        Um = U.copy(); Um[s, mu] = _expm_ah(-h * T) @ U[s, mu]
        fd = (S(Up) - S(Um)) / (2 * h)
        an = float(np.real(np.trace(P[s, mu].conj().T @ T)))
        tol = 1e-6 if inner == "f64" else 1e-6
        assert abs(fd - an) <= tol * max(1.0, abs(fd)), (fd, an)


def test_autograd_action_and_solve(env):
    torch, dw, AG = env
    dims, kappa = (4, 4, 4, 4), 0.12
    lat = dw.lattice(dims, kappa)
    U = I.gauge_field(dims, "exp", 64, 1, 0.4)
    phi = I.gaussian_spinor(dims, 64, 2)
    Ut = torch.tensor(U, device="cuda", requires_grad=True)
    pt = torch.tensor(phi, device="cuda", requires_grad=True)
    S = AG.PseudofermionAction.apply(Ut, pt, lat, _tight(dw))
    S.backward()
    X, _, _ = O.cg_normal(dims, kappa, U, phi, tol=1e-14)
    assert abs(S.item() - np.real(np.vdot(phi.reshape(-1), X.reshape(-1)))) < 1e-9 * abs(S.item())
    Gref = 2 * O.force(dims, kappa, O.dirac(dims, kappa, U, X), X)
    assert _rel(Ut.grad.cpu().numpy(), Gref) < 1e-9
    assert _rel(pt.grad.cpu().numpy(), 2 * X) < 1e-9
    # x = (D^dag D)^{-1} b with L = Re <c, x>
    c = torch.tensor(I.gaussian_spinor(dims, 64, 3), device="cuda")
    bt = torch.tensor(phi, device="cuda", requires_grad=True)
    U2 = torch.tensor(U, device="cuda", requires_grad=True)
    x = AG.CGSolve.apply(U2, bt, lat, _tight(dw))
    L = torch.vdot(c.reshape(-1), x.reshape(-1)).real
    L.backward()
    lam, _, _ = O.cg_normal(dims, kappa, U, c.cpu().numpy(), tol=1e-14)
    assert _rel(bt.grad.cpu().numpy(), lam) < 1e-9


def test_gradcheck_tiny_lattice(env):
    torch, dw, AG = env
    dims, kappa = (2, 2, 2, 2), 0.11
    lat = dw.lattice(dims, kappa)
    U = torch.tensor(I.gauge_field(dims, "exp", 65, 1, 0.4), device="cuda", requires_grad=True)
    phi = torch.tensor(I.gaussian_spinor(dims, 65, 2), device="cuda", requires_grad=True)
    p = _tight(dw)
    f = lambda u, ph: AG.PseudofermionAction.apply(u, ph, lat, p)  # noqa: E731
    assert torch.autograd.gradcheck(f, (U, phi), eps=1e-6, atol=1e-5, rtol=1e-4, fast_mode=True)
