"""Pins of the PTC (gauge-equivariant parallel-transport network) oracle:
closed forms, the adjoint of the transport, gauge equivariance and a central
finite-difference check of the analytic gradients."""
import numpy as np
import pytest

from oracle import dirac as D
from oracle import ptc as P
from synth import fields as F

DIMS = (2, 2, 2, 4)


def test_identity_path_closed_form():
    """Only the identity path, W_0 = c 1: the network multiplies by c_1 c_2 ... ."""
    u = F.gauge_field(DIMS, 1)
    cs = [0.5 + 0.2j, -1.3, 2.0j]
    ws = []
    for c in cs:
        w = np.zeros((9, 1, 1, 4, 4), complex)
        w[0, 0, 0] = c * np.eye(4)
        ws.append(w)
    net = P.PTC(u, DIMS, ws)
    r = F.odd_spinor(DIMS, 2)
    assert np.abs(net.forward(r) - np.prod(cs) * r).max() < 1e-14


def test_single_hop_matches_dirac_hopping_term():
    """A one-layer net with W_{+mu} = (1 - g_mu), W_{-mu} = (1 + g_mu) is the Wilson
    hopping term H of the Dirac oracle (restricted to odd -> odd it vanishes, so
    compare on the full lattice)."""
    u = F.gauge_field(DIMS, 3)
    w = np.zeros((9, 1, 1, 4, 4), complex)
    for mu in range(4):
        w[1 + mu, 0, 0] = np.eye(4) - D.GAMMA[mu]
        w[5 + mu, 0, 0] = np.eye(4) + D.GAMMA[mu]
    geo = D.Geometry(DIMS)
    U = D.links_flat(u)
    psi = F.spinor((geo.V, 1, 4, 3), 4)
    got = P.layer(geo, U, w, psi)[:, 0]
    ref = D.hop(geo, U, psi[:, 0])
    assert np.abs(got - ref).max() < 1e-13


def test_transport_adjoint_dot_test():
    u = F.gauge_field(DIMS, 5)
    geo = D.Geometry(DIMS)
    U = D.links_flat(u)
    a = F.spinor((geo.V, 2, 4, 3), 6)
    b = F.spinor((geo.V, 2, 4, 3), 7)
    for p in range(9):
        lhs = np.vdot(a, P.transport(geo, U, b, p))
        rhs = np.vdot(P.transport(geo, U, a, P.reverse(p)), b)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gauge_equivariance():
    dims = (4, 2, 2, 4)
    u = F.gauge_field(dims, 8)
    g = F.random_gauge_transform(dims, 9)
    ug = F.gauge_transform_links(u, g)
    ws = P.random_weights([1, 3, 2, 1], 10, scale=0.5)
    net, netg = P.PTC(u, dims, ws), P.PTC(ug, dims, ws)
    r = F.odd_spinor(dims, 11)
    gf = g.reshape(-1, 3, 3)[net.geo.odd]
    G = lambda f: np.einsum("nab,nsb->nsa", gf, f)
    assert np.abs(netg.forward(G(r)) - G(net.forward(r))).max() < 1e-12


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_gradient_finite_difference(layer):
    u = F.gauge_field(DIMS, 12)
    ws = P.random_weights([1, 2, 2, 1], 13, scale=0.8)
    net = P.PTC(u, DIMS, ws)
    r = F.odd_spinor(DIMS, 14)
    e = F.odd_spinor(DIMS, 15)
    L, grads = net.grad(r, e)
    assert abs(L - net.loss(r, e)) < 1e-14 * abs(L)
    rng = np.random.default_rng(16)
    h = 1e-6
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in ws[layer].shape)
        for unit, part in ((1.0, "re"), (1j, "im")):
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[layer][idx] += unit * h
            wm[layer][idx] -= unit * h
            fd = (P.PTC(u, DIMS, wp).loss(r, e) - P.PTC(u, DIMS, wm).loss(r, e)) / (2 * h)
            g = grads[layer][idx]
            an = 2 * (g.real if part == "re" else g.imag)
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (idx, part, fd, an)
