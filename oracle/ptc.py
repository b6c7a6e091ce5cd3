"""FP64 reference of the gauge-equivariant parallel-transport network (PTC) used
as a learned preconditioner inside flexible CG.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The network is not in the
paper (it stands in for the multigrid preconditioner of Sec. 4.1); its training
trajectory is stochastic and therefore "parity unpinned": the pins below fix the
layer, the loss and the gradients, not where training ends up.

Network (all layers linear, no activation, so the preconditioner is a linear map):
  phi_0        = the odd-site residual r embedded in the full lattice (even sites 0),
                 one channel
  phi_l^a(x)   = sum_{p in P} sum_b W_{l,p}^{ab} (T_p phi_{l-1}^b)(x)
  N(r)         = odd sites of phi_L (one channel)
with W_{l,p}^{ab} a complex 4x4 spin matrix, P = {1, +x,+y,+z,+t, -x,-y,-z,-t},
  (T_{+mu} phi)(x) = U_mu(x) phi(x+mu),  (T_{-mu} phi)(x) = U_mu(x-mu)^dag phi(x-mu)
(with the same time-boundary phase as the Dirac operator).  T_{+mu}^dag = T_{-mu}.
Loss of a training pair (r, e = A^{-1} r):  L = ||N(r) - e||^2 / ||e||^2.
Gradients are Wirtinger gradients dL/d conj(.), so the steepest-descent step is
W <- W - lr * G.
"""
from __future__ import annotations

import numpy as np

from oracle import dirac as D

# path order: 0 identity, 1..4 forward +x..+t, 5..8 backward -x..-t
PATHS = [None] + [(mu, +1) for mu in range(4)] + [(mu, -1) for mu in range(4)]


def reverse(p):
    """Index of the adjoint path: T_p^dag = T_reverse(p)."""
    return 0 if p == 0 else (p + 4 if p <= 4 else p - 4)


def transport(geo: D.Geometry, U, phi, p, bc_t=-1.0):
    """(T_p phi)(x) for a multi-channel field phi (V, C, 4, 3)."""
    if p == 0:
        return phi.copy()
    mu, d = PATHS[p]
    if d > 0:
        y = geo.fwd[mu]
        ph = np.where(geo.t_wrap_fwd, bc_t, 1.0) if mu == 3 else np.ones(geo.V)
        out = np.einsum("nab,ncsb->ncsa", U[:, mu], phi[y])
    else:
        y = geo.bwd[mu]
        ph = np.where(geo.t_wrap_bwd, bc_t, 1.0) if mu == 3 else np.ones(geo.V)
        out = np.einsum("nba,ncsb->ncsa", np.conj(U[y, mu]), phi[y])
    return ph[:, None, None, None] * out


def layer(geo, U, W, phi, bc_t=-1.0):
    """One PTC layer: W (9, Cout, Cin, 4, 4) complex, phi (V, Cin, 4, 3)."""
    out = np.zeros((geo.V, W.shape[1], 4, 3), dtype=np.complex128)
    for p in range(9):
        out += np.einsum("abst,xbtc->xasc", W[p], transport(geo, U, phi, p, bc_t))
    return out


class PTC:
    def __init__(self, u, dims, weights, bc_t=-1.0):
        """weights: list of arrays (9, Cout, Cin, 4, 4) complex, first Cin = last Cout = 1."""
        self.geo = D.Geometry(dims)
        self.U = D.links_flat(u)
        self.W = [np.asarray(w, dtype=np.complex128) for w in weights]
        self.bc_t = bc_t

    def embed(self, r_odd):
        phi = np.zeros((self.geo.V, 1, 4, 3), dtype=np.complex128)
        phi[self.geo.odd, 0] = r_odd
        return phi

    def forward(self, r_odd, keep=False):
        phis = [self.embed(r_odd)]
        for W in self.W:
            phis.append(layer(self.geo, self.U, W, phis[-1], self.bc_t))
        z = phis[-1][self.geo.odd, 0]
        return (z, phis) if keep else z

    def loss(self, r_odd, e_odd):
        z = self.forward(r_odd)
        return float(np.vdot(z - e_odd, z - e_odd).real / np.vdot(e_odd, e_odd).real)

    def grad(self, r_odd, e_odd):
        """Loss and Wirtinger gradients dL/dconj(W_l) (same shapes as the weights)."""
        z, phis = self.forward(r_odd, keep=True)
        ee = np.vdot(e_odd, e_odd).real
        L = float(np.vdot(z - e_odd, z - e_odd).real / ee)
        delta = np.zeros_like(phis[-1])
        delta[self.geo.odd, 0] = (z - e_odd) / ee
        grads = [None] * len(self.W)
        for l in range(len(self.W) - 1, -1, -1):
            W = self.W[l]
            phi_in = phis[l]
            G = np.zeros_like(W)
            back = np.zeros_like(phi_in)
            for p in range(9):
                v = transport(self.geo, self.U, phi_in, p, self.bc_t)
                G[p] = np.einsum("xasc,xbtc->abst", delta, np.conj(v))
                # d/dconj(phi): T_p^dag W_p^H delta, with T_p^dag = T_reverse(p)
                wd = np.einsum("abst,xasc->xbtc", np.conj(W[p]), delta)
                back += transport(self.geo, self.U, wd, reverse(p), self.bc_t)
            grads[l] = G
            delta = back
        return L, grads


def random_weights(channels, seed, scale=0.1):
    """Seeded complex weights for a network with the given channel list."""
    gen = np.random.Generator(np.random.Philox(key=int(seed)))
    ws = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        w = (gen.standard_normal((9, cout, cin, 4, 4)) + 1j * gen.standard_normal((9, cout, cin, 4, 4)))
        ws.append(scale * w / np.sqrt(9 * cin * 4))
    return ws
