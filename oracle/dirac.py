"""Plain FP64 definitions of the twisted-mass clover Dirac operators (Sec. 2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions (the paper fixes none of these; the readings are listed in the
design notes and pinned by tests/test_oracle_pins.py):

* lattice dims (X, Y, Z, T), each even; lexicographic site index
  lex = ((t*Z + z)*Y + y)*X + x; parity = (x+y+z+t) mod 2; the solve lives on
  ODD sites (ODD_ODD_ASYMMETRIC, Sec. 2) and odd site k has lex // 2 == k.
* spinor index (spin, colour) -> 3*spin + colour; flavour (heavy) outermost.
* chiral gamma basis:  gamma_t = [[0,-1],[-1,0]],  gamma_k = [[0,-i s_k],[i s_k,0]]
  (2x2 blocks), gamma_5 = gamma_t gamma_x gamma_y gamma_z = diag(1,1,-1,-1).
* hopping normalisation:
    M psi(x) = A(x) psi(x) + i 2 kappa mu gamma_5 psi(x) - kappa (H psi)(x)
    (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
                       + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)
    A(x) = 1 - kappa c_sw sum_{mu<nu} gamma_mu gamma_nu F_munu(x)
           (= 1 + i kappa c_sw sum_{mu<nu} sigma_munu F_munu,  sigma = (i/2)[g,g])
    F_munu = (1/8)(Q_munu - Q_munu^dag) minus 1/3 of its trace, Q_munu the sum
    of the four plaquette leaves at x in the (mu,nu) plane.
* boundary: periodic in space; antiperiodic in time as a factor bc_t on hops
  that cross t = T-1 <-> 0 (the clover uses the plain links).
* heavy doublet (eq:hQh):  M_h = M(mu=0) x 1_f + i 2 kappa mubar gamma_5 tau^3
                                  - 2 kappa epsbar tau^1.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------
# Dirac algebra
# ----------------------------------------------------------------------------
_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _blocks(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.array([
    _blocks(_Z2, -1j * _S1, 1j * _S1, _Z2),   # gamma_x
    _blocks(_Z2, -1j * _S2, 1j * _S2, _Z2),   # gamma_y
    _blocks(_Z2, -1j * _S3, 1j * _S3, _Z2),   # gamma_z
    _blocks(_Z2, -_I2, -_I2, _Z2),            # gamma_t
])
GAMMA5 = GAMMA[3] @ GAMMA[0] @ GAMMA[1] @ GAMMA[2]
ID4 = np.eye(4, dtype=np.complex128)
ID3 = np.eye(3, dtype=np.complex128)
TAU1 = _S1
TAU3 = _S3


def sigma(mu, nu):
    """sigma_munu = (i/2)[gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


def dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


# ----------------------------------------------------------------------------
# Geometry
# ----------------------------------------------------------------------------
class Geometry:
    """Neighbour tables on the (X,Y,Z,T) torus in lexicographic order."""

    def __init__(self, dims):
        X, Y, Z, T = (int(d) for d in dims)
        for d in (X, Y, Z, T):
            if d < 2 or d % 2:
                raise ValueError("every lattice extent must be even and >= 2")
        self.dims = (X, Y, Z, T)
        self.V = X * Y * Z * T
        lex = np.arange(self.V)
        x = lex % X
        y = (lex // X) % Y
        z = (lex // (X * Y)) % Z
        t = lex // (X * Y * Z)
        self.coords = np.stack([x, y, z, t])          # (4, V)
        self.parity = (x + y + z + t) % 2
        self.odd = np.nonzero(self.parity == 1)[0]   # odd[k] // 2 == k
        self.even = np.nonzero(self.parity == 0)[0]
        L = np.array(self.dims)
        self.fwd = np.empty((4, self.V), dtype=np.int64)
        self.bwd = np.empty((4, self.V), dtype=np.int64)
        for mu in range(4):
            cp = self.coords.copy()
            cp[mu] = (cp[mu] + 1) % L[mu]
            self.fwd[mu] = self._lex(cp)
            cm = self.coords.copy()
            cm[mu] = (cm[mu] - 1) % L[mu]
            self.bwd[mu] = self._lex(cm)
        # sites whose forward/backward time hop wraps around the boundary
        self.t_wrap_fwd = t == T - 1
        self.t_wrap_bwd = t == 0

    def _lex(self, c):
        X, Y, Z, _ = self.dims
        return ((c[3] * Z + c[2]) * Y + c[1]) * X + c[0]

    def embed_odd(self, psi_o):
        full = np.zeros((self.V,) + psi_o.shape[1:], dtype=np.complex128)
        full[self.odd] = psi_o
        return full

    def embed_even(self, psi_e):
        full = np.zeros((self.V,) + psi_e.shape[1:], dtype=np.complex128)
        full[self.even] = psi_e
        return full


def links_flat(u):
    """Canonical [t][z][y][x][mu][3][3] -> (V, 4, 3, 3)."""
    return np.ascontiguousarray(u).reshape(-1, 4, 3, 3)


# ----------------------------------------------------------------------------
# Hopping term
# ----------------------------------------------------------------------------
def hop(geo: Geometry, U, psi, bc_t=-1.0, sites=None):
    """(H psi)(x) at the given sites (all if None).

    psi: (V, ..., 4, 3) full-lattice field (any leading flavour axes between
    site and spin are carried along).  U: (V, 4, 3, 3).
    """
    if sites is None:
        sites = np.arange(geo.V)
    out = np.zeros((len(sites),) + psi.shape[1:], dtype=np.complex128)
    for mu in range(4):
        xf = geo.fwd[mu][sites]
        xb = geo.bwd[mu][sites]
        ph_f = np.ones(len(sites))
        ph_b = np.ones(len(sites))
        if mu == 3:
            ph_f = np.where(geo.t_wrap_fwd[sites], bc_t, 1.0)
            ph_b = np.where(geo.t_wrap_bwd[sites], bc_t, 1.0)
        pf = ID4 - GAMMA[mu]
        pb = ID4 + GAMMA[mu]
        # forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
        chi = np.einsum("nab,n...sb->n...sa", U[sites, mu], psi[xf])
        chi = np.einsum("st,n...tc->n...sc", pf, chi)
        out += ph_f.reshape((-1,) + (1,) * (psi.ndim - 1)) * chi
        # backward: (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu)
        chi = np.einsum("nab,n...sb->n...sa", dagger(U[xb, mu]), psi[xb])
        chi = np.einsum("st,n...tc->n...sc", pb, chi)
        out += ph_b.reshape((-1,) + (1,) * (psi.ndim - 1)) * chi
    return out


# ----------------------------------------------------------------------------
# Clover term
# ----------------------------------------------------------------------------
def field_strength(geo: Geometry, U, mu, nu, sites=None):
    """Clover-leaf F_munu(x) = (1/8)(Q - Q^dag) - (1/3) tr(...) at the sites."""
    if sites is None:
        sites = np.arange(geo.V)
    f, b = geo.fwd, geo.bwd
    x = sites
    xpm = f[mu][x]                 # x + mu
    xpn = f[nu][x]                 # x + nu
    xmm = b[mu][x]                 # x - mu
    xmn = b[nu][x]                 # x - nu
    xmm_pn = f[nu][xmm]            # x - mu + nu
    xmm_mn = b[nu][xmm]            # x - mu - nu
    xmn_pm = f[mu][xmn]            # x - nu + mu
    Um = U[:, mu]
    Un = U[:, nu]
    d = dagger
    leaf1 = Um[x] @ Un[xpm] @ d(Um[xpn]) @ d(Un[x])
    leaf2 = Un[x] @ d(Um[xmm_pn]) @ d(Un[xmm]) @ Um[xmm]
    leaf3 = d(Um[xmm]) @ d(Un[xmm_mn]) @ Um[xmm_mn] @ Un[xmn]
    leaf4 = d(Un[xmn]) @ Um[xmn] @ Un[xmn_pm] @ d(Um[x])
    q = leaf1 + leaf2 + leaf3 + leaf4
    F = (q - d(q)) / 8.0
    tr = np.trace(F, axis1=-2, axis2=-1)
    return F - tr[:, None, None] / 3.0 * ID3


def clover_matrix(geo: Geometry, U, kappa, csw, sites=None):
    """A(x) = 1 - kappa csw sum_{mu<nu} gamma_mu gamma_nu (x) F_munu, (n, 12, 12)."""
    if sites is None:
        sites = np.arange(geo.V)
    A = np.zeros((len(sites), 12, 12), dtype=np.complex128)
    A[:] = np.eye(12)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = field_strength(geo, U, mu, nu, sites)
            gg = GAMMA[mu] @ GAMMA[nu]
            A -= kappa * csw * np.einsum("st,nab->nsatb", gg, F).reshape(-1, 12, 12)
    return A


def apply_local(Mloc, psi):
    """Site-local matrices (n, k, k) on fields (n, ..., 4, 3) with k = size of the
    trailing (flavour, spin, colour) block."""
    n = psi.shape[0]
    return np.einsum("nij,nj->ni", Mloc, psi.reshape(n, -1)).reshape(psi.shape)


def g5(psi):
    return np.einsum("st,n...tc->n...sc", GAMMA5, psi)


def tau(psi, t):
    """Flavour matrix on a two-flavour field (n, 2, 4, 3)."""
    return np.einsum("fg,ngsc->nfsc", t, psi)


# ----------------------------------------------------------------------------
# Operators
# ----------------------------------------------------------------------------
class TwistedMassClover:
    """All operators of Sec. 2 on one gauge field, with the local blocks cached.

    mu, mubar, epsbar are the bare (mass-normalised) parameters; the operator
    uses mu_t = 2 kappa mu etc. (hopping normalisation).
    """

    def __init__(self, u, dims, kappa, csw, mu=0.0, mubar=0.0, epsbar=0.0, bc_t=-1.0,
                 sites=None):
        self.geo = Geometry(dims)
        self.U = links_flat(u)
        self.kappa = float(kappa)
        self.csw = float(csw)
        self.mu_t = 2.0 * kappa * mu
        self.mubar_t = 2.0 * kappa * mubar
        self.epsbar_t = 2.0 * kappa * epsbar
        self.bc_t = float(bc_t)
        self._A = None
        self._cache = {}

    # -- local blocks ---------------------------------------------------------
    @property
    def A(self):
        if self._A is None:
            self._A = clover_matrix(self.geo, self.U, self.kappa, self.csw)
        return self._A

    def _twist12(self, sign):
        return sign * 1j * self.mu_t * np.kron(GAMMA5, ID3)

    def local_light(self, sites, sign):
        """(A + sign i mu_t gamma_5) at the sites, (n, 12, 12)."""
        return self.A[sites] + self._twist12(sign)

    def local_heavy(self, sites, sign=+1):
        """A x 1_f + sign i mubar_t gamma_5 tau^3 - epsbar_t tau^1, (n, 24, 24).
        sign = -1 gives the operator with mubar -> -mubar."""
        n = len(sites)
        out = np.zeros((n, 24, 24), dtype=np.complex128)
        A = self.A[sites]
        out[:, :12, :12] = A
        out[:, 12:, 12:] = A
        out += sign * 1j * self.mubar_t * np.kron(TAU3, np.kron(GAMMA5, ID3))
        out -= self.epsbar_t * np.kron(TAU1, np.eye(12))
        return out

    def inv_even_light(self, sign):
        key = ("light", sign)
        if key not in self._cache:
            self._cache[key] = np.linalg.inv(self.local_light(self.geo.even, sign))
        return self._cache[key]

    def inv_even_heavy(self, sign):
        key = ("heavy", sign)
        if key not in self._cache:
            self._cache[key] = np.linalg.inv(self.local_heavy(self.geo.even, sign))
        return self._cache[key]

    # -- full-lattice operators ----------------------------------------------
    def M(self, psi, sign=+1):
        """Full M(sign*mu) on a full-lattice one-flavour field (V, 4, 3)."""
        allx = np.arange(self.geo.V)
        return apply_local(self.local_light(allx, sign), psi) \
            - self.kappa * hop(self.geo, self.U, psi, self.bc_t)

    def Q(self, psi, sign=+1):
        """Q_pm = gamma_5 M(pm mu) (Sec. 2)."""
        return g5(self.M(psi, sign))

    def M_heavy(self, psi, sign=+1):
        """Full two-flavour M_h on (V, 2, 4, 3)."""
        allx = np.arange(self.geo.V)
        return apply_local(self.local_heavy(allx, sign), psi) \
            - self.kappa * hop(self.geo, self.U, psi, self.bc_t)

    # -- even-odd Schur operators (eq:hQpm, eq:hQh) --------------------------
    def Mhat(self, psi_o, sign=+1):
        """M_oo - M_oe M_ee^{-1} M_eo on odd sites, with M_eo = -kappa H_eo."""
        geo = self.geo
        h_e = hop(geo, self.U, geo.embed_odd(psi_o), self.bc_t, geo.even)     # H_eo psi_o
        t_e = apply_local(self.inv_even_light(sign), -self.kappa * h_e)        # M_ee^-1 M_eo psi_o
        w = -self.kappa * hop(geo, self.U, geo.embed_even(t_e), self.bc_t, geo.odd)
        return apply_local(self.local_light(geo.odd, sign), psi_o) - w

    def Qhat(self, psi_o, sign=+1):
        """Q_hat_pm = gamma_5 [ (M_oo pm i mu g5) - M_oe (M_ee pm i mu g5)^-1 M_eo ]."""
        return g5(self.Mhat(psi_o, sign))

    def Mhat_heavy(self, psi_o, sign=+1):
        geo = self.geo
        h_e = hop(geo, self.U, geo.embed_odd(psi_o), self.bc_t, geo.even)
        t_e = apply_local(self.inv_even_heavy(sign), -self.kappa * h_e)
        w = -self.kappa * hop(geo, self.U, geo.embed_even(t_e), self.bc_t, geo.odd)
        return apply_local(self.local_heavy(geo.odd, sign), psi_o) - w

    def Qhat_heavy(self, psi_o, sign=+1):
        """Q_hat_h of eq:hQh on (V/2, 2, 4, 3); sign=-1 gives Q_hat_h^dagger
        (= tau^1 Q_hat_h tau^1, i.e. mubar -> -mubar)."""
        return g5(self.Mhat_heavy(psi_o, sign))

    def What(self, psi_o, rho, sign=+1):
        """Mass-preconditioned W_hat_pm(rho) = Q_hat_pm pm i rho_t (eq:hWpm), rho_t = 2 kappa rho."""
        return self.Qhat(psi_o, sign) + sign * 1j * 2.0 * self.kappa * rho * psi_o

    # -- normal operators used by the solvers --------------------------------
    def MdagM(self, psi_o):
        """M_hat^dagger M_hat = Q_hat_- Q_hat_+ (HPD)."""
        return self.Qhat(self.Qhat(psi_o, +1), -1)

    def QpQm(self, psi_o):
        """Q_hat_+ Q_hat_- (the HMC ordering)."""
        return self.Qhat(self.Qhat(psi_o, -1), +1)

    def heavy_sq(self, psi_o):
        """Q_hat_h Q_hat_h^dagger (HPD)."""
        return self.Qhat_heavy(self.Qhat_heavy(psi_o, -1), +1)

    # -- reconstruction of the even part --------------------------------------
    def schur_rhs(self, b_full, sign=+1):
        """b_hat_o = b_o - M_oe M_ee^{-1} b_e."""
        geo = self.geo
        s_e = apply_local(self.inv_even_light(sign), b_full[geo.even])
        w = -self.kappa * hop(geo, self.U, geo.embed_even(s_e), self.bc_t, geo.odd)
        return b_full[geo.odd] - w

    def reconstruct_even(self, x_o, b_full, sign=+1):
        """x_e = M_ee^{-1} (b_e - M_eo x_o)."""
        geo = self.geo
        meo = -self.kappa * hop(geo, self.U, geo.embed_odd(x_o), self.bc_t, geo.even)
        return apply_local(self.inv_even_light(sign), b_full[geo.even] - meo)

    # -- sampled evaluation at full size ---------------------------------------
    def Qhat_at(self, psi_o, odd_sites, sign=+1, heavy=False):
        """(Q_hat psi_o) at a subset of odd sites (indices into the odd list)
        without building the whole lattice's clover inverse."""
        geo = self.geo
        S = geo.odd[np.asarray(odd_sites)]
        nb = np.unique(np.concatenate([geo.fwd[m][S] for m in range(4)] +
                                      [geo.bwd[m][S] for m in range(4)]))
        full = geo.embed_odd(psi_o)
        h_e = hop(geo, self.U, full, self.bc_t, nb)
        A_nb = clover_matrix(geo, self.U, self.kappa, self.csw, nb)
        A_S = clover_matrix(geo, self.U, self.kappa, self.csw, S)
        if heavy:
            loc_nb = self._heavy_from_A(A_nb, sign)
            loc_S = self._heavy_from_A(A_S, sign)
        else:
            loc_nb = A_nb + self._twist12(sign)
            loc_S = A_S + self._twist12(sign)
        t_nb = apply_local(np.linalg.inv(loc_nb), -self.kappa * h_e)
        tfull = np.zeros_like(full)
        tfull[nb] = t_nb
        w = -self.kappa * hop(geo, self.U, tfull, self.bc_t, S)
        return g5(apply_local(loc_S, full[S]) - w)

    def _heavy_from_A(self, A, sign):
        n = A.shape[0]
        out = np.zeros((n, 24, 24), dtype=np.complex128)
        out[:, :12, :12] = A
        out[:, 12:, 12:] = A
        out += sign * 1j * self.mubar_t * np.kron(TAU3, np.kron(GAMMA5, ID3))
        out -= self.epsbar_t * np.kron(TAU1, np.eye(12))
        return out


def heavy_local_alt(A, kappa, mu_sigma, mu_delta):
    """The heavy doublet written as D_W + csw + i mu_sigma gamma_5 tau^1 + mu_delta tau^3
    (hopping normalised), (n, 24, 24): the same operator as eq:hQh up to a constant
    flavour rotation.  Used only to pin that equivalence."""
    n = A.shape[0]
    out = np.zeros((n, 24, 24), dtype=np.complex128)
    out[:, :12, :12] = A
    out[:, 12:, 12:] = A
    out += 1j * 2 * kappa * mu_sigma * np.kron(TAU1, np.kron(GAMMA5, ID3))
    out += 2 * kappa * mu_delta * np.kron(TAU3, np.eye(12))
    return out
