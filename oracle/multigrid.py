"""Aggregation-based two-level multigrid for the twisted-mass clover operator, in
FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4.1 runs the light sector's most poorly conditioned solves with a
multigrid-preconditioned outer GCR (QUDA's MG) and finds it about a hundred
times faster than mixed-precision CG at the physical quark mass.  The paper
gives no algorithmic detail of the method beyond that its library coarsens the
symmetrically even-odd preconditioned operator.  This module is the plain
textbook form of aggregation-based (Galerkin) two-level multigrid for Wilson-
type operators, applied to the full operator M of oracle.dirac:

* near-null vectors: nvec random fields smoothed by minimal-residual steps on
  M v = 0, which damp the large-eigenvalue components and leave the near
  kernel;
* aggregates: the lattice cut into blocks, each block split by chirality (the
  upper two and the lower two spins), so that the coarse operator keeps
  gamma_5-hermiticity;
* prolongator P: on every aggregate, the restrictions of the nvec vectors,
  orthonormalised (Gram-Schmidt, i.e. the QR factorisation whose R has a
  positive real diagonal, which fixes each column's phase); P^+ P = 1;
* coarse operator M_c = P^+ M P (Galerkin), nearest-neighbour on the block
  lattice;
* preconditioner: coarse-grid correction z = P M_c^-1 P^+ r followed by nu
  minimal-residual smoothing steps on M z = r;
* outer solver: GCR with that (variable) preconditioner, restarted.
"""
from __future__ import annotations

import numpy as np

from . import dirac as D


class Aggregates:
    """Block x chirality aggregates of a (X, Y, Z, T) lattice."""

    def __init__(self, geo: D.Geometry, block):
        self.geo = geo
        self.block = tuple(int(b) for b in block)
        for L, b in zip(geo.dims, self.block):
            if L % b:
                raise ValueError("block extents must divide the lattice extents")
        nb = [L // b for L, b in zip(geo.dims, self.block)]
        self.nblocks_dims = tuple(nb)
        c = geo.coords
        bc = [c[m] // self.block[m] for m in range(4)]
        self.block_of_site = ((bc[3] * nb[2] + bc[2]) * nb[1] + bc[1]) * nb[0] + bc[0]
        self.nblocks = int(np.prod(nb))
        self.sites_of_block = [np.nonzero(self.block_of_site == k)[0] for k in range(self.nblocks)]

    def block_neighbours(self, k):
        """Blocks sharing a face with block k (and k itself)."""
        nb = self.nblocks_dims
        x = [0, 0, 0, 0]
        r = k
        for m in range(4):
            x[m] = r % nb[m]
            r //= nb[m]
        out = {k}
        for m in range(4):
            for d in (-1, 1):
                y = list(x)
                y[m] = (y[m] + d) % nb[m]
                out.add(((y[3] * nb[2] + y[2]) * nb[1] + y[1]) * nb[0] + y[0])
        return out


def minimal_residual(apply_M, b, x, steps):
    """steps of minimal-residual iteration on M x = b (x updated and returned)."""
    r = b - apply_M(x)
    for _ in range(steps):
        mr = apply_M(r)
        den = np.vdot(mr, mr)
        if den == 0:
            break
        alpha = np.vdot(mr, r) / den
        x = x + alpha * r
        r = r - alpha * mr
    return x


class TwoLevelMG:
    """Two-level Galerkin multigrid preconditioner for op.M (full lattice, one flavour)."""

    def __init__(self, op: D.TwistedMassClover, block, nvec, setup_steps=30, smooth_steps=4, seed=0,
                 sign=+1, vectors=None, init=None):
        """vectors: ready near-null vectors (no setup); init: the nvec random
        starting fields of the setup (drawn from seed when None)."""
        self.op = op
        self.sign = sign
        self.agg = Aggregates(op.geo, block)
        self.nvec = nvec
        self.smooth_steps = smooth_steps
        V = op.geo.V
        if vectors is None:
            gen = np.random.default_rng(seed)
            vectors = []
            for j in range(nvec):
                if init is None:
                    v = gen.standard_normal((V, 4, 3)) + 1j * gen.standard_normal((V, 4, 3))
                else:
                    v = np.array(init[j], dtype=np.complex128).reshape(V, 4, 3)
                v = minimal_residual(self.apply, np.zeros_like(v), v, setup_steps)
                vectors.append(v / np.linalg.norm(v))
        self.vectors = vectors
        # prolongator blocks: aggregate (block k, chirality h) -> (sites, 2 spins x 3 colours, nvec)
        self.P = []
        for k in range(self.agg.nblocks):
            s = self.agg.sites_of_block[k]
            for h in range(2):
                cols = np.stack([v[s][:, 2 * h:2 * h + 2, :].reshape(-1) for v in vectors], axis=1)
                q, r = np.linalg.qr(cols)
                d = np.diag(r)
                q = q * (d / np.abs(d))[None, :]   # Gram-Schmidt: R with a positive diagonal
                self.P.append(q)
        self.ncoarse = len(self.P) * nvec
        self._Mc = None

    def apply(self, psi):
        return self.op.M(psi, self.sign)

    def prolong(self, uc):
        """Coarse vector (naggregates * nvec) -> fine field (V, 4, 3)."""
        out = np.zeros((self.op.geo.V, 4, 3), dtype=np.complex128)
        for a, q in enumerate(self.P):
            k, h = divmod(a, 2)
            s = self.agg.sites_of_block[k]
            out[s, 2 * h:2 * h + 2, :] = (q @ uc[a * self.nvec:(a + 1) * self.nvec]).reshape(len(s), 2, 3)
        return out

    def restrict(self, v):
        out = np.empty(self.ncoarse, dtype=np.complex128)
        for a, q in enumerate(self.P):
            k, h = divmod(a, 2)
            s = self.agg.sites_of_block[k]
            out[a * self.nvec:(a + 1) * self.nvec] = q.conj().T @ v[s, 2 * h:2 * h + 2, :].reshape(-1)
        return out

    def coarse_matrix(self):
        """M_c = P^+ M P, dense (ncoarse x ncoarse)."""
        if self._Mc is None:
            Mc = np.empty((self.ncoarse, self.ncoarse), dtype=np.complex128)
            e = np.zeros(self.ncoarse, dtype=np.complex128)
            for j in range(self.ncoarse):
                e[:] = 0
                e[j] = 1
                Mc[:, j] = self.restrict(self.apply(self.prolong(e)))
            self._Mc = Mc
        return self._Mc

    def coarse_gamma5(self):
        """Diagonal of the coarse gamma_5: +1 on upper-chirality aggregates, -1 on lower."""
        g = np.empty(self.ncoarse)
        for a in range(len(self.P)):
            g[a * self.nvec:(a + 1) * self.nvec] = 1.0 if a % 2 == 0 else -1.0
        return g

    def precondition(self, r):
        """z = P M_c^-1 P^+ r, then smooth_steps minimal-residual steps on M z = r."""
        uc = np.linalg.solve(self.coarse_matrix(), self.restrict(r))
        z = self.prolong(uc)
        return minimal_residual(self.apply, r, z, self.smooth_steps)


def gcr(apply_M, b, precond=None, tol=1e-10, maxiter=1000, restart=30):
    """Restarted GCR on M x = b with a (possibly variable) right preconditioner.
    Returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    it = 0
    while it < maxiter:
        ps, aps = [], []
        for _ in range(restart):
            z = precond(r) if precond is not None else r.copy()
            az = apply_M(z)
            for p, ap in zip(ps, aps):       # orthogonalise M z against the previous directions
                beta = np.vdot(ap, az)
                z = z - beta * p
                az = az - beta * ap
            na = np.linalg.norm(az)
            z, az = z / na, az / na
            alpha = np.vdot(az, r)
            x = x + alpha * z
            r = r - alpha * az
            ps.append(z)
            aps.append(az)
            it += 1
            if np.linalg.norm(r) <= tol * nb or it >= maxiter:
                return x, it
        r = b - apply_M(x)                   # restart from the true residual
    return x, it
