"""Parity of the rational approximation's applications (tm_rational_apply,
tm_rational_correction) against the FP64 oracle (oracle/rational.py).

Tolerances.  Each shifted solve stops at a true relative residual of 1e-10, so
the combination a0 b + sum a_k x_k carries an error of at most
1e-10 ||b|| sum_k a_k / (lambda_min + sigma_k) <= 1e-10 ||b|| lambda_min^-1/2,
against ||y|| >= ||b|| lambda_max^-1/2: a relative 1e-10 sqrt(cond A).  The
bound used is 10x that.  The correction series multiplies the rational
applications' errors by |p| |binom| < 1 per term.
"""
import numpy as np
import pytest

from oracle import dirac as D
from oracle import rational as RA
from oracle import solvers as S
from synth import fields as F
from tests.gpu_util import Lat, from_dev, rel, to_dev

pytestmark = pytest.mark.gpu

KAPPA, CSW = 0.1394, 1.69
HEAVY = dict(mubar=0.1246, epsbar=0.135)
LIGHT = dict(mu=0.01)


def _setup(dims, heavy, seed):
    u = F.gauge_field(dims, seed)
    kw = HEAVY if heavy else LIGHT
    op = D.TwistedMassClover(u, dims, KAPPA, CSW, **kw)
    lat = Lat(u, dims, KAPPA, CSW, **kw)
    nf = 2 if heavy else 1
    vh = int(np.prod(dims)) // 2
    apply_A = op.heavy_sq if heavy else op.MdagM
    A = S.dense_matrix(apply_A, vh, (2, 4, 3) if heavy else (4, 3))
    lam, V = np.linalg.eigh(A)
    return op, lat, nf, A, lam, V


@pytest.mark.parametrize("heavy,dims", [(True, (2, 2, 2, 4)), (False, (4, 2, 2, 4))])
@pytest.mark.parametrize("sloppy", [0, 1], ids=["f64", "f32"])
def test_rational_apply_parity(heavy, dims, sloppy):
    op, lat, nf, A, lam, V = _setup(dims, heavy, 1801)
    try:
        tm = lat.tm
        code = tm.TM_QH_SQ if heavy else tm.TM_MDAGM
        coeffs = tm.tm_rational_inv_sqrt(8, 0.9 * lam[0], 1.1 * lam[-1])
        b = F.odd_spinor(dims, 1802, nf)
        y = to_dev(np.zeros_like(b))
        infos = tm.tm_rational_apply(lat.ctx, code, coeffs, y, to_dev(b), tm.solve_params(tol=1e-10, sloppy=sloppy))
        assert all(i.status == tm.TM_OK for i in infos)
        got = from_dev(y, b.shape)
        I = np.eye(A.shape[0])
        a0, a, sigma, delta = coeffs
        ref = RA.rational_apply(lambda s, v: np.linalg.solve(A + s * I, v), a0, a, sigma, b.reshape(-1))
        bound = 1e-9 * np.sqrt(lam[-1] / lam[0])
        assert rel(got.reshape(-1), ref) < bound, rel(got.reshape(-1), ref)
        # and y is A^-1/2 b to within the approximation's delta
        exact = V @ ((V.conj().T @ b.reshape(-1)) / np.sqrt(lam))
        assert rel(got.reshape(-1), exact) <= delta + bound
    finally:
        lat.close()


@pytest.mark.parametrize("p", [-0.25, 0.5])
def test_rational_correction_parity(p):
    dims = (2, 2, 2, 4)
    op, lat, nf, A, lam, V = _setup(dims, True, 1811)
    try:
        tm = lat.tm
        coeffs = tm.tm_rational_inv_sqrt(4, 0.9 * lam[0], 1.1 * lam[-1])
        a0, a, sigma, delta = coeffs
        b = F.odd_spinor(dims, 1812, nf)
        y = to_dev(np.zeros_like(b))
        infos, napply = tm.tm_rational_correction(lat.ctx, tm.TM_QH_SQ, coeffs, p, y, to_dev(b),
                                                  tm.solve_params(tol=1e-12), series_tol=1e-13)
        got = from_dev(y, b.shape).reshape(-1)
        rl = RA.evaluate(a0, a, sigma, lam)
        zl = lam * rl * rl - 1.0
        ref = V @ ((1.0 + zl) ** p * (V.conj().T @ b.reshape(-1)))
        # the correction itself ((1 + Z)^p - 1) b is compared, not only the leading b
        assert rel(got - b.reshape(-1), ref - b.reshape(-1)) < 1e-4
        assert rel(got, ref) < 1e-10
        assert 1 <= napply <= 6
    finally:
        lat.close()


def test_rational_full_size_properties():
    """The heavy doublet at 24^3 x 48 with 12 poles on [1e-5, 1] x 1.02 lambda_max
    (the benchmark's setting): y = r(A) b satisfies <y, A y> = ||b||^2 (1 + O(delta)),
    and the heatbath field phi = (1 + Z)^-1/4 eta gives the acceptance energy
    <phi, (1 + Z)^1/2 phi> = ||eta||^2 up to the solves' accuracy."""
    import torch
    from paper_2212_06635_gb300 import tm
    dims = (24, 24, 24, 48)
    u = F.gauge_field(dims, 1002)
    lat = Lat(u, dims, 0.14, 1.69, **HEAVY)
    try:
        lmax = 1.02 * tm.tm_power_iteration(lat.ctx, tm.TM_QH_SQ, 100)
        coeffs = tm.tm_rational_inv_sqrt(12, 1e-5 * lmax, lmax)
        delta = coeffs[3]
        b = F.odd_spinor(dims, 2002, 2)
        bd = to_dev(b)
        y = torch.zeros_like(bd)
        sp = tm.solve_params(tol=1e-10, sloppy=tm.TM_F32)
        infos = tm.tm_rational_apply(lat.ctx, tm.TM_QH_SQ, coeffs, y, bd, sp)
        assert all(i.status == tm.TM_OK for i in infos)
        nb = tm.tm_field_bytes(lat.ctx, tm.TM_F64, 2)
        yn = torch.empty(nb, dtype=torch.uint8, device="cuda:0")
        an = torch.empty_like(yn)
        tm.tm_field_import(lat.ctx, tm.TM_F64, 2, yn, y)
        tm.tm_apply_Mhat(lat.ctx, tm.TM_QH_SQ, tm.TM_F64, an, yn)
        ay = torch.empty_like(bd)
        tm.tm_field_export(lat.ctx, tm.TM_F64, 2, ay, an)
        torch.cuda.synchronize()
        yAy = float(torch.dot(y.reshape(-1), ay.reshape(-1)))
        bb = float(torch.dot(bd.reshape(-1), bd.reshape(-1)))
        assert abs(yAy / bb - 1.0) <= 2.0 * delta + 1e-8, (yAy / bb - 1.0, delta)
        # solves to 1e-12 here: errors of 1e-10 sqrt(cond) per rational application
        # would move the energy by a few 1e-9
        sp12 = tm.solve_params(tol=1e-12, sloppy=tm.TM_F32)
        phi = torch.zeros_like(bd)
        _, n1 = tm.tm_rational_correction(lat.ctx, tm.TM_QH_SQ, coeffs, -0.25, phi, bd, sp12, series_tol=1e-12)
        acc = torch.zeros_like(bd)
        _, n2 = tm.tm_rational_correction(lat.ctx, tm.TM_QH_SQ, coeffs, 0.5, acc, phi, sp12, series_tol=1e-12)
        torch.cuda.synchronize()
        energy = float(torch.dot(phi.reshape(-1), acc.reshape(-1)))
        assert abs(energy / bb - 1.0) <= 1e-9, energy / bb - 1.0
        assert n1 >= 1 and n2 >= 1
    finally:
        lat.close()
