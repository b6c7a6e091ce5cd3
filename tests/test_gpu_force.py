"""Parity of the force outer products (tm_force_outer) against the FP64 oracle
(oracle/force.py), link by link.

Tolerances (relative L2 error of the force increment), derived from the
arithmetic: every product in W pairs two stored field values, each carrying
its storage rounding (relative RMS about u/sqrt(3), u the unit roundoff of the
storage), so a product carries about sqrt(2) u/sqrt(3), and sums of many such
terms with independent errors keep that relative size.
  FP32 storage  u = 2^-24: ~1e-7, plus the FP32 arithmetic and the rebuilt third
                link row (~1e-7 each); bound 1e-5.
  FP16 storage  u = 2^-11: ~4e-4; bound 3e-3 (the 16-bit operator bound).
  BF16 storage  u = 2^-8 (8-bit significand): ~3e-3 per product, the size of the
                16-bit operator bound itself; bound 6e-3.
"""
import numpy as np
import pytest

from oracle import dirac as D
from oracle import force as FO
from synth import fields as F
from tests.gpu_util import Lat, from_dev, rel, to_dev

pytestmark = pytest.mark.gpu

KAPPA, CSW, MU = 0.1394, 1.69, 0.01
FORCE_TOL = {1: 1e-5, 3: 3e-3, 2: 6e-3}
# 2^4 (neighbours coincide), one full 32-site block, a ragged tail (vh = 432),
# and several blocks (vh = 960)
DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 6, 4, 6), (8, 6, 4, 10)]


def _fields(geo, n, nf, seed):
    shp = (n, geo.V, nf, 4, 3) if nf == 2 else (n, geo.V, 4, 3)
    return F.spinor(shp, seed)


def _upload(lat, prec, nf, full, geo):
    """(even native, odd native) of one full-lattice canonical field."""
    out = []
    for sites in (geo.even, geo.odd):
        t = lat.native(prec, nf)
        lat.tm.tm_field_import(lat.ctx, prec, nf, t, to_dev(np.ascontiguousarray(full[sites])))
        out.append(t)
    return tuple(out)


def _run(lat, prec, nf, c, X, Y, geo, force0):
    import torch
    tm = lat.tm
    xs = [_upload(lat, prec, nf, X[k], geo) for k in range(len(c))]
    ys = [_upload(lat, prec, nf, Y[k], geo) for k in range(len(c))]
    fd = to_dev(force0)
    tm.tm_force_outer(lat.ctx, prec, nf, list(c), xs, ys, fd)
    torch.cuda.synchronize()
    return from_dev(fd, force0.shape)


@pytest.fixture(scope="module", params=DIMS, ids=lambda d: "x".join(map(str, d)))
def setup(request):
    dims = request.param
    u = F.gauge_field(dims, 1200 + sum(dims))
    lat = Lat(u, dims, KAPPA, CSW, mu=MU)
    geo = D.Geometry(dims)
    yield dims, geo, D.links_flat(u), lat
    lat.close()


@pytest.mark.parametrize("prec", [1, 3, 2], ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("nf", [1, 2])
def test_force_outer_parity(setup, prec, nf):
    dims, geo, U, lat = setup
    n = 3
    X = _fields(geo, n, nf, 71)
    Y = _fields(geo, n, nf, 72)
    c = [0.7, -1.3, 2.1]
    force0 = F.spinor((geo.V, 4, 3, 3), 73)      # accumulated into
    got = _run(lat, prec, nf, c, X, Y, geo, force0)
    ref = FO.hop_force(geo, U, X, Y, c, -1.0)
    assert rel(got - force0, ref) < FORCE_TOL[prec], rel(got - force0, ref)
    # the result is traceless anti-hermitian up to the accumulated start value
    inc = got - force0
    assert np.max(np.abs(inc + D.dagger(inc))) < 1e-5 * np.max(np.abs(inc))


def test_force_outer_periodic_time_and_max_pairs():
    """bc_t = +1, and the largest number of pairs one launch takes."""
    from paper_2212_06635_gb300 import tm
    dims = (4, 4, 2, 6)
    u = F.gauge_field(dims, 1301)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU, bc_t=1)
    try:
        geo = D.Geometry(dims)
        n = tm.TM_FORCE_MAXN
        X = _fields(geo, n, 1, 81)
        Y = _fields(geo, n, 1, 82)
        c = list(np.random.default_rng(83).uniform(-1, 1, n))
        force0 = np.zeros((geo.V, 4, 3, 3), dtype=np.complex128)
        got = _run(lat, 1, 1, c, X, Y, geo, force0)
        ref = FO.hop_force(geo, D.links_flat(u), X, Y, c, 1.0)
        assert rel(got, ref) < FORCE_TOL[1]
    finally:
        lat.close()


def test_force_outer_edge_cases(setup):
    """n = 0 leaves the force unchanged; bad arguments fail on the host."""
    import torch
    dims, geo, U, lat = setup
    tm = lat.tm
    force0 = F.spinor((geo.V, 4, 3, 3), 91)
    fd = to_dev(force0)
    tm.tm_force_outer(lat.ctx, 1, 2, [], [], [], fd)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(fd, force0.shape), force0)
    pair = (lat.native(1, 1), lat.native(1, 1))
    for args in ((0, 1, [1.0], [pair], [pair], fd),               # FP64 fields
                 (1, 3, [1.0], [pair], [pair], fd),               # nflavour 3
                 (1, 1, [1.0] * 33, [pair] * 33, [pair] * 33, fd),  # too many pairs
                 (1, 1, [1.0], [pair], [(pair[0], 0)], fd),       # null field
                 (1, 1, [1.0], [pair], [pair], force0.ctypes.data)):  # host force
        assert tm.tm_force_outer(lat.ctx, *args, check=False) == tm.TM_ERR_ARG


def test_force_outer_needs_current_gauge():
    from paper_2212_06635_gb300 import tm
    import torch
    dims = (4, 4, 4, 4)
    u = F.gauge_field(dims, 1401)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU)
    try:
        tm.tm_gauge_load(lat.ctx, np.ascontiguousarray(u), 2.0)     # clover now stale
        pair = (lat.native(1, 1), lat.native(1, 1))
        fd = torch.zeros(int(np.prod(dims)) * 4 * 18, dtype=torch.float64, device="cuda:0")
        assert tm.tm_force_outer(lat.ctx, 1, 1, [1.0], [pair], [pair], fd, check=False) == tm.TM_ERR_STALE
    finally:
        lat.close()


def test_force_outer_full_size_sampled():
    """The launch the benchmark times: heavy doublet, 12 pairs, FP32 fields, on
    24^3 x 48, checked at sampled links (including time links across the
    boundary) against the oracle evaluated at those links only."""
    import torch
    from paper_2212_06635_gb300 import tm
    dims = (24, 24, 24, 48)
    n, nf = 12, 2
    u = F.gauge_field(dims, 1002)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU)
    try:
        geo = D.Geometry(dims)
        U = D.links_flat(u)
        rng = np.random.default_rng(5)
        T = dims[3]
        last = np.nonzero(geo.coords[3] == T - 1)[0]
        sites = np.unique(np.concatenate([rng.integers(0, geo.V, 96), rng.choice(last, 32, replace=False),
                                          [0, geo.V - 1]]))
        c = list(rng.uniform(0.1, 2.0, n))
        W = np.zeros((len(sites), 4, 3, 3), dtype=np.complex128)
        xs, ys = [], []
        for k in range(n):
            Xk = _fields(geo, 1, nf, 1100 + k)
            Yk = _fields(geo, 1, nf, 1200 + k)
            xs.append(_upload(lat, 1, nf, Xk[0], geo))
            ys.append(_upload(lat, 1, nf, Yk[0], geo))
            W += FO.outer_W(geo, U, Xk, Yk, [c[k]], -1.0, sites)
            del Xk, Yk
        ref = FO.project_ta(np.einsum("nmab,nmbc->nmac", U[sites], W))
        fd = torch.zeros(geo.V * 4 * 18, dtype=torch.float64, device="cuda:0")
        tm.tm_force_outer(lat.ctx, 1, nf, c, xs, ys, fd)
        torch.cuda.synchronize()
        got = from_dev(fd, (geo.V, 4, 3, 3))[sites]
        assert rel(got, ref) < FORCE_TOL[1], rel(got, ref)
    finally:
        lat.close()


def _schur_codes(tm, heavy, sign):
    if heavy:
        return (tm.TM_QH, tm.TM_QH_DAG) if sign > 0 else (tm.TM_QH_DAG, tm.TM_QH)
    return (tm.TM_QHAT_PLUS, tm.TM_QHAT_MINUS) if sign > 0 else (tm.TM_QHAT_MINUS, tm.TM_QHAT_PLUS)


@pytest.mark.parametrize("prec", [0, 1, 3], ids=["f64", "f32", "f16"])
@pytest.mark.parametrize("heavy,sign", [(False, +1), (False, -1), (True, +1), (True, -1)])
def test_apply_even_parity(prec, heavy, sign):
    """tm_apply_even = M_ee(s)^-1 H_eo on the even sites (the even pass alone)."""
    from tests.gpu_util import tol
    dims = (6, 4, 4, 6)
    u = F.gauge_field(dims, 1611)
    kw = dict(mubar=0.1246, epsbar=0.135) if heavy else dict(mu=MU)
    op = D.TwistedMassClover(u, dims, KAPPA, CSW, **kw)
    lat = Lat(u, dims, KAPPA, CSW, **kw)
    try:
        tm = lat.tm
        nf = 2 if heavy else 1
        psi = F.odd_spinor(dims, 1612, nf)
        src = to_dev(psi)
        a = lat.native(prec, nf)
        o = lat.native(prec, nf)
        tm.tm_field_import(lat.ctx, prec, nf, a, src)
        tm.tm_apply_even(lat.ctx, _schur_codes(tm, heavy, sign)[0], prec, o, a)
        out = src.clone()
        tm.tm_field_export(lat.ctx, prec, nf, out, o)
        got = from_dev(out, psi.shape)
        geo = op.geo
        h_e = D.hop(geo, op.U, geo.embed_odd(psi), op.bc_t, geo.even)
        inv = op.inv_even_heavy(sign) if heavy else op.inv_even_light(sign)
        ref = D.apply_local(inv, h_e)
        assert rel(got, ref) < tol(prec), rel(got, ref)
    finally:
        lat.close()


@pytest.mark.parametrize("heavy,sign", [(False, +1), (False, -1), (True, +1), (True, -1)])
def test_schur_force_through_the_library(heavy, sign):
    """The hopping force of Re <a, Q_hat_s b> computed by the library alone: the
    even reconstructions R_s b and R_-s a from tm_apply_even, then one
    tm_force_outer pair with g5 on Y and weight -kappa^2, against the oracle's
    pair (pinned by finite differences in test_oracle_force.py)."""
    import torch
    dims = (6, 4, 4, 6)
    u = F.gauge_field(dims, 1601)
    kw = dict(mubar=0.1246, epsbar=0.135) if heavy else dict(mu=MU)
    op = D.TwistedMassClover(u, dims, KAPPA, CSW, **kw)
    lat = Lat(u, dims, KAPPA, CSW, **kw)
    try:
        tm = lat.tm
        nf = 2 if heavy else 1
        prec = 1
        a = F.odd_spinor(dims, 1602, nf)
        b = F.odd_spinor(dims, 1603, nf)
        na, nb, ra, rb = (lat.native(prec, nf) for _ in range(4))
        tm.tm_field_import(lat.ctx, prec, nf, na, to_dev(a))
        tm.tm_field_import(lat.ctx, prec, nf, nb, to_dev(b))
        cs, cms = _schur_codes(tm, heavy, sign)
        tm.tm_apply_even(lat.ctx, cs, prec, rb, nb)
        tm.tm_apply_even(lat.ctx, cms, prec, ra, na)
        fd = torch.zeros(op.geo.V * 4 * 18, dtype=torch.float64, device="cuda:0")
        tm.tm_force_outer(lat.ctx, prec, nf, [-KAPPA ** 2], [(rb, nb)], [(ra, na)], fd, gamma5_y=True)
        torch.cuda.synchronize()
        got = from_dev(fd, (op.geo.V, 4, 3, 3))
        X, Y = FO.schur_pairs(op, a, b, sign, heavy)
        ref = FO.hop_force(op.geo, op.U, X[None], Y[None], [-KAPPA ** 2], op.bc_t)
        assert rel(got, ref) < FORCE_TOL[1], rel(got, ref)
    finally:
        lat.close()
