"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Every pin here checks the oracle against something other than itself: the
Dirac algebra, identities stated in Sec. 2, closed forms (free field, abelian
flux), symmetries (gauge covariance, gamma_5-hermiticity), tree-level O(a)
improvement of the clover term, and brute-force dense solves.
"""
import numpy as np
import pytest

from oracle import dirac as D
from oracle import solvers as S
from synth import fields as F

KAPPA, CSW, MU = 0.1394, 1.69, 0.01


def _op(dims, seed=1000, **kw):
    u = F.gauge_field(dims, seed)
    args = dict(kappa=KAPPA, csw=CSW, mu=MU)
    args.update(kw)
    return D.TwistedMassClover(u, dims, **args), u


def _full_spinor(dims, seed, nflav=1):
    V = int(np.prod(dims))
    return F.spinor((V, 4, 3) if nflav == 1 else (V, nflav, 4, 3), seed)


# ---------------------------------------------------------------------------
def test_gamma_algebra():
    G = D.GAMMA
    for a in range(4):
        assert np.allclose(G[a], G[a].conj().T)
        for b in range(4):
            assert np.allclose(G[a] @ G[b] + G[b] @ G[a], 2 * (a == b) * np.eye(4))
    assert np.allclose(D.GAMMA5, np.diag([1, 1, -1, -1]))
    for a in range(4):
        assert np.allclose(D.GAMMA5 @ G[a], -G[a] @ D.GAMMA5)
    # sigma_munu commutes with gamma_5 (clover is block diagonal in chirality)
    for a in range(4):
        for b in range(4):
            assert np.allclose(D.sigma(a, b) @ D.GAMMA5, D.GAMMA5 @ D.sigma(a, b))


def test_clover_block_structure_and_hermiticity():
    op, _ = _op((4, 4, 4, 4))
    A = op.A
    assert np.allclose(A, np.conj(np.swapaxes(A, 1, 2)), atol=1e-14)
    # zero between chirality + (spins 0,1) and chirality - (spins 2,3)
    assert np.abs(A[:, :6, 6:]).max() < 1e-15
    assert np.abs(A[:, 6:, :6]).max() < 1e-15


# P1: M(mu)^dagger = gamma_5 M(-mu) gamma_5 (Sec. 2, (Q+)^dagger = Q-) ------
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_P1_gamma5_hermiticity_full_and_schur(dims):
    op, _ = _op(dims)
    phi = _full_spinor(dims, 11)
    psi = _full_spinor(dims, 12)
    lhs = S.dot(phi, op.Q(psi, +1))
    rhs = S.dot(op.Q(phi, -1), psi)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)
    phi_o = F.odd_spinor(dims, 13)
    psi_o = F.odd_spinor(dims, 14)
    lhs = S.dot(phi_o, op.Qhat(psi_o, +1))
    rhs = S.dot(op.Qhat(phi_o, -1), psi_o)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # M_hat^dagger M_hat = Q_hat_- Q_hat_+ is hermitian positive
    a = S.dot(psi_o, op.MdagM(psi_o))
    assert abs(a.imag) <= 1e-13 * abs(a) and a.real > 0


# P2: det(Q+ Q-) = det(Q^2 + mu^2) via the operator identity Q+Q- = Q^2 + mu_t^2
def test_P2_QpQm_equals_Q2_plus_mu2():
    dims = (4, 4, 4, 4)
    op, u = _op(dims)
    op0 = D.TwistedMassClover(u, dims, KAPPA, CSW, mu=0.0)
    psi = _full_spinor(dims, 21)
    lhs = op.Q(op.Q(psi, -1), +1)
    rhs = op0.Q(op0.Q(psi)) + op.mu_t ** 2 * psi
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(lhs).max()


# P3: free field plane waves -------------------------------------------------
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 1, 2)])
def test_P3_free_field_plane_wave(n):
    dims = (4, 6, 4, 8)
    X, Y, Z, T = dims
    u = F.unit_gauge(dims)
    kappa, mu = 0.13, 0.05
    op = D.TwistedMassClover(u, dims, kappa, 1.7, mu=mu)
    geo = op.geo
    L = np.array(dims)
    p = 2 * np.pi * np.array(n, dtype=float) / L
    p[3] += np.pi / T                                   # antiperiodic time
    chi = F.spinor((4, 3), 31)
    phase = np.exp(1j * (p[:, None] * geo.coords).sum(0))
    psi = phase[:, None, None] * chi[None]
    a = 1 - 2 * kappa * np.cos(p).sum()
    Mp = a * np.eye(4) + 2j * kappa * sum(D.GAMMA[m] * np.sin(p[m]) for m in range(4)) \
        + 2j * kappa * mu * D.GAMMA5
    expect = phase[:, None, None] * (Mp @ chi)[None]
    got = op.M(psi)
    assert np.abs(got - expect).max() < 1e-13
    # closed-form inverse
    den = a * a + 4 * kappa ** 2 * (np.sin(p) ** 2).sum() + 4 * kappa ** 2 * mu ** 2
    Minv = (a * np.eye(4) - 2j * kappa * sum(D.GAMMA[m] * np.sin(p[m]) for m in range(4))
            - 2j * kappa * mu * D.GAMMA5) / den
    assert np.allclose(Minv @ Mp, np.eye(4), atol=1e-14)
    # the clover term vanishes for unit links
    assert np.abs(op.A - np.eye(12)).max() < 1e-15


# P4 / P5: pure gauge and gauge covariance ----------------------------------
def test_P4_pure_gauge():
    dims = (4, 4, 4, 4)
    g = F.random_gauge_transform(dims, 41)
    u = F.pure_gauge(g)
    op = D.TwistedMassClover(u, dims, KAPPA, CSW, mu=MU)
    assert np.abs(op.A - np.eye(12)).max() < 1e-13
    op1 = D.TwistedMassClover(F.unit_gauge(dims), dims, KAPPA, CSW, mu=MU)
    psi = _full_spinor(dims, 42)
    gf = g.reshape(-1, 3, 3)
    Gpsi = np.einsum("nab,nsb->nsa", gf, psi)
    assert np.abs(op.M(Gpsi) - np.einsum("nab,nsb->nsa", gf, op1.M(psi))).max() < 1e-12


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 4, 4)])
def test_P5_gauge_covariance(dims):
    u = F.gauge_field(dims, 51)
    g = F.random_gauge_transform(dims, 52)
    ug = F.gauge_transform_links(u, g)
    gf = g.reshape(-1, 3, 3)
    kw = dict(kappa=KAPPA, csw=CSW, mu=MU, mubar=0.1246, epsbar=0.135)
    op = D.TwistedMassClover(u, dims, **kw)
    opg = D.TwistedMassClover(ug, dims, **kw)
    psi = _full_spinor(dims, 53)
    G = lambda f, sites: np.einsum("nab,n...sb->n...sa", gf[sites], f)
    allx = np.arange(op.geo.V)
    assert np.abs(opg.M(G(psi, allx)) - G(op.M(psi), allx)).max() < 1e-12
    odd = op.geo.odd
    psi_o = F.odd_spinor(dims, 54)
    assert np.abs(opg.Qhat(G(psi_o, odd)) - G(op.Qhat(psi_o), odd)).max() < 1e-12
    psi2 = F.odd_spinor(dims, 55, 2)
    assert np.abs(opg.Qhat_heavy(G(psi2, odd)) - G(op.Qhat_heavy(psi2), odd)).max() < 1e-12


# P6: abelian flux closed form of the clover-leaf field strength -------------
@pytest.mark.parametrize("plane,n", [((0, 1), 1), ((1, 3), 2), ((2, 3), -1)])
def test_P6_abelian_flux_field_strength(plane, n):
    dims = (4, 6, 4, 8)
    mu, nu = plane
    u = F.abelian_flux(dims, mu, nu, n)
    geo = D.Geometry(dims)
    Uf = D.links_flat(u)
    phi = 2 * np.pi * n / (dims[mu] * dims[nu])
    expect = 1j * np.sin(phi) * np.diag([1.0, -1.0, 0.0])
    for a in range(4):
        for b in range(a + 1, 4):
            Fab = D.field_strength(geo, Uf, a, b)
            if (a, b) == (mu, nu):
                assert np.abs(Fab - expect).max() < 1e-14
            else:
                assert np.abs(Fab).max() < 1e-14


def test_P6_abelian_flux_trace_subtraction():
    """Charges (1,1,-2): the leaf difference has a trace, which F_munu drops."""
    dims = (4, 4, 2, 2)
    u = F.abelian_flux(dims, 0, 1, 1, charges=(1.0, 1.0, -2.0))
    phi = 2 * np.pi / 16
    raw = np.sin(phi * np.array([1.0, 1.0, -2.0]))
    expect = 1j * np.diag(raw - raw.sum() / 3)
    Fxy = D.field_strength(D.Geometry(dims), D.links_flat(u), 0, 1)
    assert np.abs(Fxy - expect).max() < 1e-14


def test_P6b_clover_sign_tree_level_improvement():
    """Tree-level O(a) improvement fixes the sign of the clover term: in a
    constant abelian field the would-be zero modes of the Wilson operator are
    shifted by O(a F) from the free value 1 - 8 kappa; the clover term with
    c_sw = 1 cancels that shift, leaving O(a^2 F^2).  (Charge +1 colour only.)"""
    dims = (8, 8, 2, 2)
    kappa = 0.1
    u = F.abelian_flux(dims, 0, 1, 1)
    shifts = {}
    for csw in (1.0, 0.0):
        op = D.TwistedMassClover(u, dims, kappa, csw, mu=0.0, bc_t=1.0)
        V = op.geo.V

        def colour0(v):
            full = np.zeros((V, 4, 3), dtype=np.complex128)
            full[..., 0] = v
            return op.M(full)[..., 0]
        M = S.dense_matrix(colour0, V, (4,))
        ev = np.linalg.eigvals(M)
        lo = ev[np.argmin(ev.real)]
        shifts[csw] = abs(lo - (1 - 8 * kappa))
    assert shifts[0.0] > 5e-3
    assert shifts[1.0] < 0.05 * shifts[0.0]


# P7: even-odd Schur solve == full solve --------------------------------------
def test_P7_schur_vs_full_solve():
    dims = (2, 2, 2, 2)
    op, _ = _op(dims, seed=71)
    V = op.geo.V
    b = _full_spinor(dims, 72)
    Mfull = S.dense_matrix(lambda v: op.M(v), V, (4, 3))
    x = np.linalg.solve(Mfull, b.ravel()).reshape(V, 4, 3)
    bh = op.schur_rhs(b)
    # M_hat x_o = b_hat  <=>  Q_hat_+ x_o = g5 b_hat  <=>  (Q-Q+) x_o = Q- g5 b_hat
    rhs = op.Qhat(D.g5(bh), -1)
    xo, _ = S.cg(op.MdagM, rhs, tol=1e-13, maxiter=5000)
    assert np.abs(xo - x[op.geo.odd]).max() < 1e-10 * np.abs(x).max()
    xe = op.reconstruct_even(xo, b)
    assert np.abs(xe - x[op.geo.even]).max() < 1e-10 * np.abs(x).max()


# P8: brute force dense solve of the normal Schur system -----------------------
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_P8_dense_bruteforce(dims):
    op, _ = _op(dims, seed=81)
    vh = op.geo.V // 2
    b = F.odd_spinor(dims, 82)
    Qp = S.dense_matrix(lambda v: op.Qhat(v, +1), vh, (4, 3))
    A = Qp.conj().T @ Qp                             # M_hat^dag M_hat = Q-Q+
    x_dense = np.linalg.solve(A, b.ravel())
    x_cg, _ = S.cg(op.MdagM, b, tol=1e-12, maxiter=5000)
    assert np.linalg.norm(x_cg.ravel() - x_dense) <= 1e-10 * np.linalg.norm(x_dense)
    # Q_hat_- as a dense matrix is the adjoint of Q_hat_+
    Qm = S.dense_matrix(lambda v: op.Qhat(v, -1), vh, (4, 3))
    assert np.abs(Qm - Qp.conj().T).max() < 1e-13


# P9, P10: heavy doublet -------------------------------------------------------
def test_P9_heavy_epsbar0_reduces_to_light_pair():
    dims = (4, 4, 4, 4)
    u = F.gauge_field(dims, 91)
    mubar = 0.1246
    oph = D.TwistedMassClover(u, dims, 0.14, CSW, mubar=mubar, epsbar=0.0)
    opl = D.TwistedMassClover(u, dims, 0.14, CSW, mu=mubar)
    psi2 = F.odd_spinor(dims, 92, 2)
    out = oph.Qhat_heavy(psi2)
    assert np.abs(out[:, 0] - opl.Qhat(psi2[:, 0], +1)).max() < 1e-13
    assert np.abs(out[:, 1] - opl.Qhat(psi2[:, 1], -1)).max() < 1e-13


def test_P9b_heavy_block_inverse_closed_form():
    """(A + i s m tau3 - e tau1)^-1 = [[(A - i s m) D, e D], [e D, (A + i s m) D]]
    with D = (A^2 + m^2 - e^2)^-1, per chirality block s = +-1."""
    op, _ = _op((4, 4, 4, 4), mubar=0.1246, epsbar=0.135, mu=0.0)
    A = op.A[op.geo.even]
    m, e = op.mubar_t, op.epsbar_t
    inv = op.inv_even_heavy(+1)
    for s, sl in ((+1, slice(0, 6)), (-1, slice(6, 12))):
        a = A[:, sl, sl]
        Dm = np.linalg.inv(a @ a + (m * m - e * e) * np.eye(6))
        top = (a - 1j * s * m * np.eye(6)) @ Dm
        bot = (a + 1j * s * m * np.eye(6)) @ Dm
        sl_u = slice(sl.start, sl.stop)
        sl_d = slice(12 + sl.start, 12 + sl.stop)
        assert np.abs(inv[:, sl_u, sl_u] - top).max() < 1e-13
        assert np.abs(inv[:, sl_d, sl_d] - bot).max() < 1e-13
        assert np.abs(inv[:, sl_u, sl_d] - e * Dm).max() < 1e-13
        assert np.abs(inv[:, sl_d, sl_u] - e * Dm).max() < 1e-13


def test_P10_heavy_adjoint_is_tau1_conjugation():
    dims = (4, 4, 4, 4)
    op, _ = _op(dims, mu=0.0, mubar=0.1246, epsbar=0.135)
    phi = F.odd_spinor(dims, 101, 2)
    psi = F.odd_spinor(dims, 102, 2)
    lhs = S.dot(phi, op.Qhat_heavy(psi, +1))
    rhs = S.dot(op.Qhat_heavy(phi, -1), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    t1 = lambda f: D.tau(f, D.TAU1)
    assert np.abs(op.Qhat_heavy(psi, -1) - t1(op.Qhat_heavy(t1(psi), +1))).max() < 1e-13


def test_P10b_heavy_forms_unitarily_equivalent():
    """eq:hQh's i mubar g5 tau3 - epsbar tau1 and the i mu_s g5 tau1 + mu_d tau3
    form are related by the constant flavour rotation W = tau1 (tau1+tau3)/sqrt2."""
    op, _ = _op((2, 2, 2, 4), mu=0.0, mubar=0.1246, epsbar=0.135)
    sites = np.arange(op.geo.V)
    Lp = op.local_heavy(sites, +1)
    La = D.heavy_local_alt(op.A, op.kappa, 0.1246, 0.135)
    W = np.kron(D.TAU1 @ (D.TAU1 + D.TAU3) / np.sqrt(2), np.eye(12))
    assert np.abs(W @ Lp @ W.conj().T - La).max() < 1e-14


# P11: multishift CG == independent CG per shift -------------------------------
def test_P11_multishift_vs_independent_cg():
    dims = (4, 4, 4, 4)
    op, _ = _op(dims, seed=111, mu=0.0, mubar=0.1246, epsbar=0.135)
    b = F.odd_spinor(dims, 112, 2)
    shifts = [1e-4, 3e-3, 0.05, 0.7]
    xs, _ = S.multishift_cg(op.heavy_sq, b, shifts, tol=1e-11, maxiter=5000)
    for s, x in zip(shifts, xs):
        A = lambda v, s=s: op.heavy_sq(v) + s * v
        xi, _ = S.cg(A, b, tol=1e-12, maxiter=5000)
        assert np.linalg.norm((x - xi).ravel()) <= 1e-9 * np.linalg.norm(xi.ravel())


def test_power_iteration_closed_form():
    d = np.linspace(0.1, 3.0, 50)
    lam = S.power_iteration(lambda v: d[:, None] * v, F.spinor((50, 1), 5), iters=2000)
    assert abs(lam - 3.0) < 1e-6


def test_W_hat_identity_on_full_operator():
    """eq:hWpm: W+ W- = Q+ Q- + 2 mu rho + rho^2 holds exactly for the full
    operator (Q_pm = Q pm i mu_t); W_pm = Q_pm pm i rho_t."""
    dims = (4, 4, 4, 4)
    op, _ = _op(dims)
    rho_t = 2 * KAPPA * 0.05
    psi = _full_spinor(dims, 121)
    Wp = lambda v: op.Q(v, +1) + 1j * rho_t * v
    Wm = lambda v: op.Q(v, -1) - 1j * rho_t * v
    lhs = Wp(Wm(psi))
    rhs = op.Q(op.Q(psi, -1), +1) + (2 * op.mu_t * rho_t + rho_t ** 2) * psi
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(lhs).max()


def test_sampled_evaluation_matches_whole_lattice():
    dims = (4, 4, 2, 6)
    op, _ = _op(dims, mubar=0.1246, epsbar=0.135)
    psi = F.odd_spinor(dims, 131)
    psi2 = F.odd_spinor(dims, 132, 2)
    s = np.array([0, 3, 17, 40, op.geo.V // 2 - 1])
    for sign in (+1, -1):
        assert np.abs(op.Qhat_at(psi, s, sign) - op.Qhat(psi, sign)[s]).max() < 1e-13
        assert np.abs(op.Qhat_at(psi2, s, sign, heavy=True)
                      - op.Qhat_heavy(psi2, sign)[s]).max() < 1e-13
