"""Pins of the rational approximation and its correction term (oracle/rational.py).

* Optimality: by Chebyshev's alternation theorem the best type-(n, n)
  approximation's relative error equioscillates at 2n + 2 points of the
  interval, so the partial-fraction form's error is sampled on a fine grid and
  its alternation counted.
* Scaling: the coefficients of [s lo, s hi] follow from those of [lo, hi].
* Matrix functions: r(A) b from shifted dense solves lies within delta of
  A^-1/2 b computed by eigendecomposition, and the binomial series of (1 + Z)^p
  matches the matrix power.  The heatbath and acceptance factors cancel exactly.
"""
import numpy as np
import pytest

from oracle import dirac as D
from oracle import rational as RA
from oracle import solvers as S
from synth import fields as F


def _alternations(a0, a, sigma, lo, hi):
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 400001))
    err = np.sqrt(x) * RA.evaluate(a0, a, sigma, x) - 1.0
    peak = np.abs(err).max()
    near = np.nonzero(np.abs(err) >= 0.98 * peak)[0]
    signs = np.sign(err[near])
    runs = 1 + int(np.count_nonzero(np.diff(signs) != 0))
    return runs, peak


@pytest.mark.parametrize("n,lo,hi", [(3, 1e-2, 1.0), (4, 1e-3, 2.0), (6, 1e-4, 3.0), (8, 1e-5, 1.0),
                                     (12, 2.7e-5, 2.7)])
def test_zolotarev_equioscillates(n, lo, hi):
    a0, a, sigma, delta = RA.zolotarev_inv_sqrt(n, lo, hi)
    runs, peak = _alternations(a0, a, sigma, lo, hi)
    assert runs == 2 * n + 2, runs
    assert abs(peak - delta) <= 1e-3 * delta
    assert np.all(sigma > 0) and np.all(a > 0) and a0 > 0


def test_zolotarev_scaling_and_convergence():
    a0, a, s, d = RA.zolotarev_inv_sqrt(8, 1e-4, 1.0)
    b0, b, t, e = RA.zolotarev_inv_sqrt(8, 3e-4, 3.0)
    assert abs(e - d) < 1e-12
    assert np.allclose(b0, a0 / np.sqrt(3.0), rtol=1e-12)
    assert np.allclose(b, a * np.sqrt(3.0), rtol=1e-12)
    assert np.allclose(t, 3.0 * s, rtol=1e-12)
    deltas = [RA.zolotarev_inv_sqrt(n, 1e-5, 1.0)[3] for n in (4, 6, 8, 10, 12)]
    assert all(d2 < 0.2 * d1 for d1, d2 in zip(deltas, deltas[1:]))


@pytest.fixture(scope="module")
def dense_heavy():
    dims = (2, 2, 2, 4)
    u = F.gauge_field(dims, 1701)
    op = D.TwistedMassClover(u, dims, 0.1394, 1.69, mubar=0.1246, epsbar=0.135)
    vh = int(np.prod(dims)) // 2
    A = S.dense_matrix(op.heavy_sq, vh, (2, 4, 3))
    lam, V = np.linalg.eigh(A)
    b = F.odd_spinor(dims, 1702, 2).reshape(-1)
    return A, lam, V, b


def test_rational_apply_within_delta(dense_heavy):
    A, lam, V, b = dense_heavy
    a0, a, sigma, delta = RA.zolotarev_inv_sqrt(6, 0.9 * lam[0], 1.1 * lam[-1])
    I = np.eye(len(b))
    y = RA.rational_apply(lambda s, v: np.linalg.solve(A + s * I, v), a0, a, sigma, b)
    exact = V @ ((V.conj().T @ b) / np.sqrt(lam))
    err = np.linalg.norm(y - exact) / np.linalg.norm(exact)
    assert err <= delta * 1.0001
    assert err > 1e-3 * delta          # the approximation error is visible, not hidden


@pytest.mark.parametrize("p", [-0.25, 0.5])
def test_correction_series_and_cancellation(dense_heavy, p):
    A, lam, V, b = dense_heavy
    a0, a, sigma, delta = RA.zolotarev_inv_sqrt(4, 0.9 * lam[0], 1.1 * lam[-1])
    rl = RA.evaluate(a0, a, sigma, lam)
    zl = lam * rl * rl - 1.0                      # eigenvalues of Z = A r(A)^2 - 1
    assert np.max(np.abs(zl)) <= 2.0 * delta + delta ** 2
    Z = (V * zl) @ V.conj().T
    y, napply = RA.binomial_series(p, lambda v: Z @ v, b)
    exact = V @ ((1.0 + zl) ** p * (V.conj().T @ b))
    assert np.linalg.norm(y - exact) <= 1e-13 * np.linalg.norm(exact)
    assert 1 <= napply <= 6
    if p == 0.5:
        phi, _ = RA.binomial_series(-0.25, lambda v: Z @ v, b)
        acc, _ = RA.binomial_series(0.5, lambda v: Z @ v, phi)
        assert abs(np.vdot(phi, acc).real - np.vdot(b, b).real) <= 1e-12 * np.vdot(b, b).real


def test_golden_zolotarev_coefficients():
    """The stored coefficients (tests/golden/zolotarev_n12_1e-5.txt, written by
    tests/golden/make_golden.py from this oracle) still come out, so a change of
    the oracle's arithmetic shows here; and the stored approximation itself
    equioscillates at 2n + 2 points."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "zolotarev_n12_1e-5.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    a0 = float(rows[0][0])
    a = np.array([float(r[0]) for r in rows[1:13]])
    sigma = np.array([float(r[1]) for r in rows[1:13]])
    delta = float(rows[13][0])
    b0, b, s, d = RA.zolotarev_inv_sqrt(12, 1e-5, 1.0)
    assert abs(b0 - a0) <= 1e-13 * a0
    assert np.allclose(b, a, rtol=1e-12) and np.allclose(s, sigma, rtol=1e-12)
    assert abs(d - delta) <= 1e-9 * delta
    runs, peak = _alternations(a0, a, sigma, 1e-5, 1.0)
    assert runs == 26 and abs(peak - delta) <= 1e-3 * delta
