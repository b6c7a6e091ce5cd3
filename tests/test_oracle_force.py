"""Pins of the force outer products (oracle/force.py) against the mathematics.

The force is the derivative of S(U) = sum_k c_k Re <Y_k, H[U] X_k> along
su(3) directions of the links.  The pins differentiate S numerically through
oracle.dirac.hop (itself pinned against the free-field closed form, gauge
covariance and gamma_5-hermiticity in test_oracle_pins.py) and check the
covariance of F under gauge transformations.
"""
import numpy as np
import pytest

from oracle import dirac as D
from oracle import force as FO
from synth import fields as F


def _expm_anti(omega):
    """exp(omega) for a stack of anti-hermitian 3x3 matrices, via eigh of -i omega."""
    lam, vec = np.linalg.eigh(-1j * omega)
    return np.einsum("...ab,...b,...cb->...ac", vec, np.exp(1j * lam), np.conj(vec))


def _random_su3_algebra(shape, seed):
    """i sum_a h_a lambda_a / 2, h_a ~ N(0,1): anti-hermitian and traceless."""
    gen = np.random.default_rng(seed)
    h = gen.standard_normal(shape + (8,))
    lam = F.gell_mann()
    return 0.5j * np.einsum("...a,aij->...ij", h, lam)


def _setup(dims, n, nf, seed):
    geo = D.Geometry(dims)
    U = D.links_flat(F.gauge_field(dims, 1000 + seed))
    shp = (n, geo.V, nf, 4, 3) if nf == 2 else (n, geo.V, 4, 3)
    X = F.spinor(shp, 2000 + seed)
    Y = F.spinor(shp, 3000 + seed)
    c = np.random.default_rng(seed).uniform(0.2, 2.0, n)
    return geo, U, X, Y, c


def _fd(geo, U, X, Y, c, bc_t, omega, h=1e-4):
    """Central difference of S(exp(t omega) U) at t = 0."""
    up = np.einsum("nmab,nmbc->nmac", _expm_anti(h * omega), U)
    um = np.einsum("nmab,nmbc->nmac", _expm_anti(-h * omega), U)
    return (FO.action(geo, up, X, Y, c, bc_t) - FO.action(geo, um, X, Y, c, bc_t)) / (2 * h)


@pytest.mark.parametrize("dims,nf,bc_t", [((4, 4, 4, 4), 2, -1.0), ((4, 4, 4, 4), 1, 1.0),
                                          ((2, 4, 2, 4), 2, -1.0), ((4, 2, 6, 2), 1, -1.0)])
def test_force_is_derivative_of_hopping_form(dims, nf, bc_t):
    """dS/dt along random su(3) directions on all links = sum Re tr(omega F).
    Central differences with h = 1e-4 are exact up to h^2/6 |omega|^2 ~ 1e-8
    relative (S is linear in each link)."""
    geo, U, X, Y, c = _setup(dims, 3, nf, 11)
    Fo = FO.hop_force(geo, U, X, Y, c, bc_t)
    omega = _random_su3_algebra((geo.V, 4), 7)
    pred = float(np.real(np.einsum("nmab,nmba->", omega, Fo)))
    fd = _fd(geo, U, X, Y, c, bc_t, omega)
    assert abs(pred - fd) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("mu,t_boundary", [(0, False), (1, False), (2, False), (3, False), (3, True)])
def test_force_single_link(mu, t_boundary):
    """The derivative along one link alone, including a time link across the
    antiperiodic boundary (where W carries the phase bc_t)."""
    dims = (4, 4, 4, 6)
    geo, U, X, Y, c = _setup(dims, 2, 2, 23)
    bc_t = -1.0
    T = dims[3]
    cand = np.nonzero(geo.coords[3] == (T - 1 if t_boundary else 2))[0]
    x = int(cand[5])
    omega = np.zeros((geo.V, 4, 3, 3), dtype=np.complex128)
    omega[x, mu] = _random_su3_algebra((), 31 + mu)
    Fo = FO.hop_force(geo, U, X, Y, c, bc_t, sites=[x])
    pred = float(np.real(np.trace(omega[x, mu] @ Fo[0, mu])))
    fd = _fd(geo, U, X, Y, c, bc_t, omega)
    assert abs(pred - fd) <= 1e-8 * max(1.0, abs(fd))
    # the boundary phase matters: with periodic time the derivative differs
    if t_boundary:
        Fp = FO.hop_force(geo, U, X, Y, c, 1.0, sites=[x])
        assert abs(np.real(np.trace(omega[x, mu] @ Fp[0, mu])) - pred) > 1e-3 * abs(pred)


def test_force_gauge_covariance():
    """U -> g(x) U g(x+mu)^+, X -> g X, Y -> g Y  gives  F_mu(x) -> g(x) F_mu(x) g(x)^+."""
    dims = (4, 4, 2, 4)
    geo, U, X, Y, c = _setup(dims, 2, 2, 41)
    g = F.random_gauge_transform(dims, 43).reshape(geo.V, 3, 3)
    Ug = D.links_flat(F.gauge_transform_links(U.reshape(dims[::-1] + (4, 3, 3)),
                                              g.reshape(dims[::-1] + (3, 3))))
    Xg = np.einsum("vab,nvfsb->nvfsa", g, X)
    Yg = np.einsum("vab,nvfsb->nvfsa", g, Y)
    F0 = FO.hop_force(geo, U, X, Y, c)
    F1 = FO.hop_force(geo, Ug, Xg, Yg, c)
    want = np.einsum("vab,vmbc,vdc->vmad", g, F0, np.conj(g))
    assert np.max(np.abs(F1 - want)) <= 1e-12 * np.max(np.abs(F0))


def test_force_algebra_and_sites():
    """F is traceless anti-hermitian, linear in the weights, and the sampled
    evaluation agrees with the full one."""
    geo, U, X, Y, c = _setup((4, 4, 4, 4), 3, 1, 5)
    Fo = FO.hop_force(geo, U, X, Y, c)
    assert np.max(np.abs(Fo + D.dagger(Fo))) < 1e-13
    assert np.max(np.abs(np.trace(Fo, axis1=-2, axis2=-1))) < 1e-13
    F1 = FO.hop_force(geo, U, X[:1], Y[:1], c[:1])
    F2 = FO.hop_force(geo, U, X[1:], Y[1:], c[1:])
    assert np.max(np.abs(F1 + F2 - Fo)) < 1e-12
    s = np.array([0, 17, 100, geo.V - 1])
    assert np.max(np.abs(FO.hop_force(geo, U, X, Y, c, sites=s) - Fo[s])) < 1e-13


@pytest.mark.parametrize("heavy,sign", [(False, +1), (False, -1), (True, +1), (True, -1)])
def test_schur_hopping_force(heavy, sign):
    """The pair built by schur_pairs gives, with weight -kappa^2, the derivative of
    Re <a, Q_hat_sign b> along su(3) directions of every link, the clover term
    held at its value for the unperturbed links (its own link dependence is not
    part of the hopping force)."""
    dims = (4, 4, 2, 4)
    kappa, csw = 0.1394, 1.69
    u = F.gauge_field(dims, 1501)
    kw = dict(mubar=0.1246, epsbar=0.135) if heavy else dict(mu=0.01)
    op = D.TwistedMassClover(u, dims, kappa, csw, **kw)
    nf = 2 if heavy else 1
    a = F.odd_spinor(dims, 1502, nf)
    b = F.odd_spinor(dims, 1503, nf)
    X, Y = FO.schur_pairs(op, a, b, sign, heavy)
    Fo = FO.hop_force(op.geo, op.U, X[None], Y[None], [-kappa ** 2], op.bc_t)
    omega = _random_su3_algebra((op.geo.V, 4), 1504)
    pred = float(np.real(np.einsum("nmab,nmba->", omega, Fo)))

    def form(t):
        ut = np.einsum("nmab,nmbc->nmac", _expm_anti(t * omega), op.U).reshape(u.shape)
        opt = D.TwistedMassClover(ut, dims, kappa, csw, **kw)
        opt._A = op.A                      # clover held fixed
        q = opt.Qhat_heavy(b, sign) if heavy else opt.Qhat(b, sign)
        return float(np.real(np.vdot(a, q)))

    h = 1e-4
    fd = (form(h) - form(-h)) / (2 * h)
    assert abs(pred - fd) <= 1e-7 * max(1.0, abs(fd)), (pred, fd)
