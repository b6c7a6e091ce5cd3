"""Fermion-force outer products of the hopping term on every link, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4.3 ("Efficiency") names the force of the rational-approximation
monomials as the part its runs left on the CPU: it needs colour outer products
of several two-flavour spinors, one pair per shift of the multishift solve.
This module is the plain definition of that step.

Definition.  Take pairs of full-lattice fields (X_k, Y_k), k = 0 .. n-1, with
one or two flavours, and real weights c_k.  The form

    S(U) = sum_k c_k Re <Y_k, H[U] X_k>

(H the hopping term of oracle.dirac, time-boundary phase included) depends on
the link U_mu(x) only through Re tr(U_mu(x) W_mu(x)), where

    W_mu(x) = ph_mu(x) sum_k c_k sum_flavour sum_spin
                [ X_k(x+mu)_s  (x)  ((1 - g_mu) Y_k(x))_s^*
                + ((1 + g_mu) Y_k(x+mu))_s  (x)  X_k(x)_s^* ]

with (a (x) b^*)_{ij} = a_i conj(b_j) over colour, and ph_mu(x) = bc_t on the
time links that cross t = T-1 -> 0 (1 elsewhere).  The first term comes from
the forward hop at x, the second from the backward hop at x+mu, which uses
U_mu(x)^dagger.  Moving U_mu(x) -> exp(t Omega) U_mu(x), Omega in su(3),
changes S at the rate Re tr(Omega U W) = Re tr(Omega F) with

    F_mu(x) = T_A[ U_mu(x) W_mu(x) ],   T_A[Z] = (Z - Z^+)/2 - tr(Z - Z^+)/6,

the traceless anti-hermitian part.  F is the force field returned here.  The
clover term's dependence on the links (its own force) is not part of this step.

Pinned in tests/test_oracle_force.py against the derivative of S taken by
finite differences through oracle.dirac.hop, and against gauge covariance.
"""
from __future__ import annotations

import numpy as np

from . import dirac as D


def _as_fields(F):
    """(n, V, [nf,] 4, 3) -> (n, V, nf, 4, 3)."""
    F = np.asarray(F)
    if F.ndim == 4:
        F = F[:, :, None]
    return F


def outer_W(geo: D.Geometry, U, X, Y, coeffs, bc_t=-1.0, sites=None):
    """W_mu(x) at the given base sites x (all if None): (len(sites), 4, 3, 3).

    X, Y: (n, V, [nf,] 4, 3) full-lattice fields; coeffs: n reals.
    """
    X = _as_fields(X)
    Y = _as_fields(Y)
    if sites is None:
        sites = np.arange(geo.V)
    sites = np.asarray(sites)
    W = np.zeros((len(sites), 4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        xf = geo.fwd[mu][sites]
        ph = np.ones(len(sites))
        if mu == 3:
            ph = np.where(geo.t_wrap_fwd[sites], bc_t, 1.0)
        pm = D.ID4 - D.GAMMA[mu]
        pp = D.ID4 + D.GAMMA[mu]
        for k, c in enumerate(coeffs):
            # forward hop at x: X(x+mu) (x) ((1 - g_mu) Y(x))^*
            py = np.einsum("st,nftc->nfsc", pm, Y[k][sites])
            t1 = np.einsum("nfsb,nfsa->nba", X[k][xf], np.conj(py))
            # backward hop at x+mu (through U_mu(x)^dagger): ((1 + g_mu) Y(x+mu)) (x) X(x)^*
            py = np.einsum("st,nftc->nfsc", pp, Y[k][xf])
            t2 = np.einsum("nfsa,nfsb->nab", py, np.conj(X[k][sites]))
            W[:, mu] += c * ph[:, None, None] * (t1 + t2)
    return W


def project_ta(Z):
    """Traceless anti-hermitian part of a stack of 3x3 matrices."""
    A = 0.5 * (Z - D.dagger(Z))
    tr = np.trace(A, axis1=-2, axis2=-1) / 3.0
    return A - tr[..., None, None] * D.ID3


def hop_force(geo: D.Geometry, U, X, Y, coeffs, bc_t=-1.0, sites=None):
    """F_mu(x) = T_A[U_mu(x) W_mu(x)] at the given base sites: (len(sites), 4, 3, 3)."""
    if sites is None:
        sites = np.arange(geo.V)
    sites = np.asarray(sites)
    W = outer_W(geo, U, X, Y, coeffs, bc_t, sites)
    return project_ta(np.einsum("nmab,nmbc->nmac", U[sites], W))


def action(geo: D.Geometry, U, X, Y, coeffs, bc_t=-1.0):
    """S(U) = sum_k c_k Re <Y_k, H[U] X_k> (used to pin the force by differentiation)."""
    X = _as_fields(X)
    Y = _as_fields(Y)
    s = 0.0
    for k, c in enumerate(coeffs):
        hx = D.hop(geo, U, X[k], bc_t)
        s += c * float(np.real(np.vdot(Y[k], hx)))
    return s


def schur_pairs(op: D.TwistedMassClover, a_o, b_o, sign=+1, heavy=False):
    """Full-lattice fields (X, Y) whose hopping force, with weight -kappa^2, is the
    derivative of Re <a, Q_hat_sign b> along the links with the clover term held
    fixed (Q_hat of eq:hQpm, or of eq:hQh when heavy).

    Q_hat = g5 [M_oo - kappa^2 H_oe M_ee^-1 H_eo], so varying the two hops gives
        Re <g5 a, dH_oe R_s b> + Re <(M_ee^-1)^+ H_oe^+ g5 a, dH_eo b>,  R_s = M_ee(s)^-1 H_eo,
    with (M_ee(s)^-1)^+ = M_ee(-s)^-1 (the twist flips sign), H^+ = g5 H g5 and g5
    commuting with M_ee, so the second even field is g5 R_-s a.  The two pairs
    live on opposite parities, so one pair carries both:
        X = (R_s b on even sites, b on odd sites),  Y = g5 (R_-s a, a).
    """
    geo = op.geo

    def R(psi_o, s):
        h_e = D.hop(geo, op.U, geo.embed_odd(psi_o), op.bc_t, geo.even)
        inv = op.inv_even_heavy(s) if heavy else op.inv_even_light(s)
        return D.apply_local(inv, h_e)

    X = np.zeros((geo.V,) + b_o.shape[1:], dtype=np.complex128)
    Y = np.zeros_like(X)
    X[geo.even] = R(b_o, sign)
    X[geo.odd] = b_o
    Y[geo.even] = D.g5(R(a_o, -sign))
    Y[geo.odd] = D.g5(a_o)
    return X, Y
