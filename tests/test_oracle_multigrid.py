"""Pins of the two-level multigrid oracle (oracle/multigrid.py).

* The prolongator is orthonormal (P^+ P = 1), and the coarse-grid correction
  is exact on the coarse space: P M_c^-1 P^+ M P u = P u.
* The coarse operator inherits gamma_5-hermiticity from the fine one
  (M(mu)^+ = g5 M(-mu) g5, pinned in test_oracle_pins.py), because the
  aggregates split by chirality: M_c(mu)^+ = G5 M_c(-mu) G5.
* The coarse operator couples only aggregates in the same or face-neighbouring
  blocks: the hopping term is nearest-neighbour.
* Degenerate case: one-site aggregates with as many vectors as an aggregate has
  components make P unitary, the coarse solve the exact inverse, and GCR
  converge in one step.
* Gain: multigrid-preconditioned GCR needs far fewer iterations than plain GCR.
"""
import numpy as np
import pytest

from oracle import dirac as D
from oracle import multigrid as MG
from synth import fields as F

KAPPA, CSW, MU = 0.1394, 1.69, 0.01


def _op(dims, seed, mu=MU):
    u = F.gauge_field(dims, seed)
    return D.TwistedMassClover(u, dims, KAPPA, CSW, mu=mu)


@pytest.fixture(scope="module")
def mg44():
    op = _op((4, 4, 4, 4), 1911)
    return op, MG.TwoLevelMG(op, (2, 2, 2, 2), 4, setup_steps=10, seed=1)


def test_prolongator_orthonormal_and_exact_on_coarse_space(mg44):
    op, mg = mg44
    gen = np.random.default_rng(2)
    u = gen.standard_normal(mg.ncoarse) + 1j * gen.standard_normal(mg.ncoarse)
    pu = mg.prolong(u)
    assert abs(np.linalg.norm(pu) - np.linalg.norm(u)) < 1e-12 * np.linalg.norm(u)
    assert np.allclose(mg.restrict(pu), u, atol=1e-12)
    back = mg.prolong(np.linalg.solve(mg.coarse_matrix(), mg.restrict(mg.apply(pu))))
    assert np.linalg.norm(back - pu) < 1e-11 * np.linalg.norm(pu)


def test_coarse_gamma5_hermiticity(mg44):
    op, mg = mg44
    mgm = MG.TwoLevelMG(op, (2, 2, 2, 2), 4, sign=-1, vectors=mg.vectors)
    Mp = mg.coarse_matrix()
    Mm = mgm.coarse_matrix()
    g = mg.coarse_gamma5()
    lhs = Mp.conj().T
    rhs = g[:, None] * Mm * g[None, :]
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(Mp))
    assert np.max(np.abs(Mp - Mm)) > 1e-3 * np.max(np.abs(Mp))    # the twist does enter


def test_coarse_operator_nearest_neighbour(mg44):
    op, mg = mg44
    Mc = mg.coarse_matrix()
    nv = mg.nvec
    scale = np.max(np.abs(Mc))
    checked = 0
    for a in range(2 * mg.agg.nblocks):
        ka = a // 2
        near = mg.agg.block_neighbours(ka)
        for b in range(2 * mg.agg.nblocks):
            blk = Mc[a * nv:(a + 1) * nv, b * nv:(b + 1) * nv]
            if b // 2 not in near:
                assert np.max(np.abs(blk)) < 1e-13 * scale
                checked += 1
    assert checked > 0
    # and face-neighbouring blocks do couple (block 1 is block 0's x neighbour)
    assert 1 in mg.agg.block_neighbours(0)
    assert np.max(np.abs(Mc[0:2 * nv, 2 * nv:4 * nv])) > 1e-3 * scale


def test_full_coarse_space_is_exact():
    op = _op((2, 2, 2, 2), 1921)
    mg = MG.TwoLevelMG(op, (1, 1, 1, 1), 6, setup_steps=5, smooth_steps=0, seed=4)
    assert mg.ncoarse == 16 * 12
    b = F.spinor((16, 4, 3), 1922)
    x, it = MG.gcr(mg.apply, b, mg.precondition, tol=1e-12)
    assert it == 1
    assert np.linalg.norm(b - mg.apply(x)) <= 1e-12 * np.linalg.norm(b)


def test_multigrid_gain():
    dims = (4, 4, 4, 8)
    op = _op(dims, 1901)
    b = F.spinor((int(np.prod(dims)), 4, 3), 1902)
    mg = MG.TwoLevelMG(op, (2, 2, 2, 4), 8, setup_steps=20, smooth_steps=4, seed=3)
    x0, it0 = MG.gcr(mg.apply, b, None, tol=1e-8, maxiter=3000)
    x1, it1 = MG.gcr(mg.apply, b, mg.precondition, tol=1e-8, maxiter=500)
    for x in (x0, x1):
        assert np.linalg.norm(b - mg.apply(x)) <= 1.01e-8 * np.linalg.norm(b)
    assert it1 * 4 < it0, (it0, it1)


def test_prolongator_is_gram_schmidt(mg44):
    """Each aggregate's columns are the Gram-Schmidt orthonormalisation of the
    restricted near-null vectors: P_a^+ V_a is upper triangular with a positive
    real diagonal (the unique QR factor with that property), so the columns'
    phases are fixed by the vectors alone."""
    op, mg = mg44
    for a, q in enumerate(mg.P):
        k, h = divmod(a, 2)
        s = mg.agg.sites_of_block[k]
        cols = np.stack([v[s][:, 2 * h:2 * h + 2, :].reshape(-1) for v in mg.vectors], axis=1)
        r = q.conj().T @ cols
        assert np.allclose(q.conj().T @ q, np.eye(mg.nvec), atol=1e-12)
        assert np.max(np.abs(np.tril(r, -1))) < 1e-12 * np.max(np.abs(r))
        d = np.diag(r)
        assert np.all(d.real > 0) and np.max(np.abs(d.imag)) < 1e-12 * np.max(np.abs(d))
        assert np.linalg.norm(q @ r - cols) < 1e-12 * np.linalg.norm(cols)
