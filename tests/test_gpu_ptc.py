"""The gauge-equivariant parallel-transport network (learned preconditioner) on
the GPU against the FP64 oracle: forward pass, loss and gradient parity,
closed forms, equivariance, checkpointing, training progress and the gain of
the trained network inside flexible CG over CG without it.

Tolerances: activations, weights and transported fields are rounded to BF16
(unit roundoff 2^-9 = 2e-3) once per layer each, so an L-layer forward pass is
bounded by about 3 L roundings: 2e-2 relative L2 for 4 layers; gradients pass
through twice as many roundings: 5e-2.
"""
import numpy as np
import pytest

from oracle import ptc as P
from oracle import solvers as S
from oracle import dirac as D
from synth import fields as F
from tests.gpu_util import Lat, from_dev, rel, to_dev

pytestmark = pytest.mark.gpu

KAPPA, CSW, MU = 0.14, 1.69, 0.005
FWD_TOL, GRAD_TOL = 2e-2, 5e-2


def _flat(ws):
    return np.concatenate([w.ravel() for w in ws])


def _net(tm, channels, ws=None):
    net = tm.tm_ptc_create(channels)
    if ws is not None:
        tm.tm_ptc_set_weights(net, _flat(ws))
    return net


def _apply(tm, lat, net, r):
    import torch
    src = to_dev(r)
    a = lat.native(tm.TM_F32, 1)
    o = lat.native(tm.TM_F32, 1)
    tm.tm_field_import(lat.ctx, tm.TM_F32, 1, a, src)
    tm.tm_ptc_apply(net, lat.ctx, o, a)
    tm.tm_ptc_sync(net)   # raises if a layer's bounded tensor-core wait ran out
    out = src.clone()
    tm.tm_field_export(lat.ctx, tm.TM_F32, 1, out, o)
    torch.cuda.synchronize()
    return from_dev(out, r.shape)


# 10x10x12x18: 21600 sites = 168 full tiles of 128 and a ragged tail of 96,
# more tiles than SMs, so blocks loop over several tiles
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (10, 10, 12, 18)])
def test_forward_matches_oracle(dims):
    u = F.gauge_field(dims, 21)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU)
    tm = lat.tm
    chans = [1, 8, 8, 8, 1]
    ws = P.random_weights(chans, 22, scale=1.0)
    net = _net(tm, chans, ws)
    try:
        r = F.odd_spinor(dims, 23)
        assert rel(_apply(tm, lat, net, r), P.PTC(u, dims, ws).forward(r)) < FWD_TOL
        assert np.allclose(tm.tm_ptc_get_weights(net), _flat(ws), rtol=1e-6, atol=1e-7)
    finally:
        tm.tm_ptc_destroy(net)
        lat.close()


def test_two_hop_layers_give_hopping_term_squared():
    """Two layers with W_{+mu} = 1 - g_mu, W_{-mu} = 1 + g_mu reproduce H H on odd sites."""
    dims = (4, 4, 2, 6)
    u = F.gauge_field(dims, 24)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU)
    tm = lat.tm
    w = np.zeros((9, 1, 1, 4, 4), complex)
    for mu in range(4):
        w[1 + mu, 0, 0] = np.eye(4) - D.GAMMA[mu]
        w[5 + mu, 0, 0] = np.eye(4) + D.GAMMA[mu]
    net = _net(tm, [1, 1, 1], [w, w])
    try:
        r = F.odd_spinor(dims, 25)
        geo = D.Geometry(dims)
        U = D.links_flat(u)
        hh = D.hop(geo, U, D.hop(geo, U, geo.embed_odd(r)))[geo.odd]
        assert rel(_apply(tm, lat, net, r), hh) < FWD_TOL
    finally:
        tm.tm_ptc_destroy(net)
        lat.close()


def test_init_identity_closed_form():
    dims = (4, 4, 4, 4)
    u = F.gauge_field(dims, 26)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU)
    tm = lat.tm
    net = _net(tm, [1, 8, 8, 1])
    try:
        tm.tm_ptc_init(net, scale=0.5, noise=0.0, seed=1)
        r = F.odd_spinor(dims, 27)
        assert rel(_apply(tm, lat, net, r), 0.125 * r) < 1e-2
    finally:
        tm.tm_ptc_destroy(net)
        lat.close()


def test_gradient_matches_oracle():
    dims = (4, 4, 2, 4)
    u = F.gauge_field(dims, 28)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU)
    tm = lat.tm
    chans = [1, 4, 4, 1]
    ws = P.random_weights(chans, 29, scale=1.0)
    net = _net(tm, chans, ws)
    try:
        r = F.odd_spinor(dims, 30)
        e = F.odd_spinor(dims, 31)
        L_ref, g_ref = P.PTC(u, dims, ws).grad(r, e)
        L, g = tm.tm_ptc_grad(net, lat.ctx, to_dev(r), to_dev(e))
        assert abs(L - L_ref) < FWD_TOL * L_ref
        off = 0
        for gl in g_ref:
            n = gl.size
            assert rel(g[off:off + n], gl.ravel()) < GRAD_TOL
            off += n
    finally:
        tm.tm_ptc_destroy(net)
        lat.close()


def test_equivariance_on_gpu():
    dims = (4, 4, 2, 4)
    u = F.gauge_field(dims, 32)
    g = F.random_gauge_transform(dims, 33)
    ug = F.gauge_transform_links(u, g)
    lat, latg = Lat(u, dims, KAPPA, CSW, mu=MU), Lat(ug, dims, KAPPA, CSW, mu=MU)
    tm = lat.tm
    chans = [1, 2, 2, 1]
    net = _net(tm, chans, P.random_weights(chans, 34, scale=1.0))
    try:
        r = F.odd_spinor(dims, 35)
        gf = g.reshape(-1, 3, 3)[D.Geometry(dims).odd]
        G = lambda f: np.einsum("nab,nsb->nsa", gf, f)
        assert rel(_apply(tm, latg, net, G(r)), G(_apply(tm, lat, net, r))) < FWD_TOL
    finally:
        tm.tm_ptc_destroy(net)
        lat.close()
        latg.close()


def test_save_load_roundtrip(tmp_path):
    from paper_2212_06635_gb300 import tm
    chans = [1, 4, 1]
    a = _net(tm, chans, P.random_weights(chans, 36))
    b = _net(tm, chans)
    try:
        tm.tm_ptc_save(a, tmp_path / "net.bin")
        tm.tm_ptc_load(b, tmp_path / "net.bin")
        assert np.array_equal(tm.tm_ptc_get_weights(a), tm.tm_ptc_get_weights(b))
        c = _net(tm, [1, 2, 1])
        with pytest.raises(tm.TMError):
            tm.tm_ptc_load(c, tmp_path / "net.bin")
        tm.tm_ptc_destroy(c)
    finally:
        tm.tm_ptc_destroy(a)
        tm.tm_ptc_destroy(b)


def test_training_reduces_loss_and_helps_fcg():
    """Train on solver-generated pairs of two configurations, then solve on a
    third: the trained network must cut the loss and the FCG iteration count
    below CG's; the FP64 true residual of every solve is re-checked by the oracle."""
    dims = (8, 8, 8, 8)
    lats = [Lat(F.gauge_field(dims, 40 + k), dims, KAPPA, CSW, mu=MU) for k in range(3)]
    tm = lats[0].tm
    net = _net(tm, [1, 8, 8, 1])
    try:
        tm.tm_ptc_init(net, scale=0.5, noise=0.02, seed=7)
        losses = tm.tm_ptc_train(net, [lats[0].ctx, lats[1].ctx], tm.TM_MDAGM, npairs=400, batch=4, lr=3e-3,
                                 seed=5000)
        assert np.all(np.isfinite(losses))
        assert losses[-40:].mean() < 0.8 * losses[:40].mean()
        u = F.gauge_field(dims, 42)
        op = D.TwistedMassClover(u, dims, KAPPA, CSW, mu=MU)
        b = F.odd_spinor(dims, 43)
        x = to_dev(np.zeros_like(b))
        info = tm.tm_solve_fcg(lats[2].ctx, tm.TM_MDAGM, net, tm.solve_params(tol=1e-10), x, to_dev(b))
        assert S.rel_residual(op.MdagM, from_dev(x, b.shape), b) <= 1.05e-10
        x.zero_()
        cg = tm.tm_solve_cg(lats[2].ctx, tm.TM_MDAGM, tm.solve_params(tol=1e-10, sloppy=tm.TM_F32), x, to_dev(b))
        assert info.iters < cg.iters, (info.iters, cg.iters)
    finally:
        tm.tm_ptc_destroy(net)
        for l in lats:
            l.close()


def test_bounded_wait_runs_out_and_leaves_the_context_usable():
    """The PTC kernels bound every mbarrier wait; a wait that nothing completes
    must end after its bound with the abort flag set, and later work must run."""
    import time
    import torch
    from paper_2212_06635_gb300 import tm
    t0 = time.perf_counter()
    assert tm.tm_wait_selftest(2e-3) == 1
    assert time.perf_counter() - t0 < 5.0
    x = torch.arange(1024, dtype=torch.float64, device="cuda")
    assert float((x * 2).sum()) == 1023 * 1024


def test_network_follows_a_new_context_at_a_reused_address():
    """The network caches a transport-link field per context.  Destroying a
    context and creating the next one (whose address the allocator may reuse,
    with the same gauge generation and boundary phase) must not leave the
    previous gauge field's links in use: each forward pass matches the oracle on
    its own field."""
    dims = (4, 4, 2, 4)
    chans = [1, 8, 1]
    ws = P.random_weights(chans, 41, scale=1.0)
    net = None
    try:
        for seed in (42, 43, 44):
            u = F.gauge_field(dims, seed)
            lat = Lat(u, dims, KAPPA, CSW, mu=MU)
            try:
                if net is None:
                    net = _net(lat.tm, chans, ws)
                r = F.odd_spinor(dims, seed + 100)
                assert rel(_apply(lat.tm, lat, net, r), P.PTC(u, dims, ws).forward(r)) < FWD_TOL
            finally:
                lat.close()
    finally:
        if net is not None:
            lat.tm.tm_ptc_destroy(net)


def test_gradients_alternating_between_two_live_contexts():
    """One network used on two contexts in turn (A, B, A): the transport-link
    field follows the context of each call, so every loss and gradient matches
    the oracle on that context's own gauge field."""
    dims = (4, 4, 2, 4)
    chans = [1, 8, 1]
    ws = P.random_weights(chans, 51, scale=1.0)
    ua, ub = F.gauge_field(dims, 52), F.gauge_field(dims, 53)
    la, lb = Lat(ua, dims, KAPPA, CSW, mu=MU), Lat(ub, dims, KAPPA, CSW, mu=MU)
    tm = la.tm
    net = _net(tm, chans, ws)
    try:
        r = F.odd_spinor(dims, 54)
        e = F.odd_spinor(dims, 55)
        for lat, u in ((la, ua), (lb, ub), (la, ua)):
            L_ref, g_ref = P.PTC(u, dims, ws).grad(r, e)
            L, g = tm.tm_ptc_grad(net, lat.ctx, to_dev(r), to_dev(e))
            assert abs(L - L_ref) < FWD_TOL * L_ref
            assert rel(g, np.concatenate([x.ravel() for x in g_ref])) < GRAD_TOL
    finally:
        tm.tm_ptc_destroy(net)
        la.close()
        lb.close()
