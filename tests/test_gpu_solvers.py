"""Solvers through the C ABI against the FP64 oracle: FP64 CG, mixed-precision
CG with reliable updates (Sec. 4.1), multishift CG with shift-by-shift
refinement (Sec. 4.2), batched solves, power iteration, and error paths.
Every returned solution is re-checked by the oracle's own FP64 residual."""
import numpy as np
import pytest

from oracle import dirac as D
from oracle import solvers as S
from synth import fields as F
from tests.gpu_util import Lat, from_dev, rel, to_dev

pytestmark = pytest.mark.gpu

CSW = 1.69


def _lat(dims, seed, kappa=0.1394, mu=0.01, mubar=0.0, epsbar=0.0):
    u = F.gauge_field(dims, seed)
    op = D.TwistedMassClover(u, dims, kappa, CSW, mu=mu, mubar=mubar, epsbar=epsbar)
    return op, Lat(u, dims, kappa, CSW, mu=mu, mubar=mubar, epsbar=epsbar)


def test_fp64_cg_4x4_to_1e12():
    op, lat = _lat((4, 4, 4, 4), 1000)
    tm = lat.tm
    try:
        b = F.odd_spinor((4, 4, 4, 4), 2000)
        x = to_dev(np.zeros_like(b))
        info = tm.tm_solve_cg(lat.ctx, tm.TM_MDAGM, tm.solve_params(tol=1e-12), x, to_dev(b))
        xs = from_dev(x, b.shape)
        assert S.rel_residual(op.MdagM, xs, b) < 1.05e-12
        assert info.true_rel_res < 1e-12
        xo, _ = S.cg(op.MdagM, b, tol=1e-13, maxiter=5000)
        assert rel(xs, xo) < 1e-9
        _, k = S.cg(op.MdagM, b, tol=1e-12, maxiter=5000)   # same stopping rule
        assert abs(info.iters - k) <= 3
    finally:
        lat.close()


@pytest.mark.parametrize("sloppy", [1, 3, 2], ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("graph", [1, 0], ids=["graph", "stream"])
def test_mixed_precision_cg_8x8(sloppy, graph):
    dims = (8, 8, 8, 8)
    op, lat = _lat(dims, 1100, kappa=0.1400, mu=0.005)
    tm = lat.tm
    try:
        b = F.odd_spinor(dims, 2100)
        x = to_dev(np.zeros_like(b))
        sp = tm.solve_params(tol=1e-10, sloppy=sloppy, use_graph=graph)
        info = tm.tm_solve_cg(lat.ctx, tm.TM_MDAGM, sp, x, to_dev(b))
        res = S.rel_residual(op.MdagM, from_dev(x, b.shape), b)
        assert res <= 1.05e-10 and info.true_rel_res <= 1e-10
        assert info.reliable_updates >= 1
    finally:
        lat.close()


def test_fp64_reliable_updates_option():
    """tm_solve_params.fp64_updates = 1 recomputes every reliable-update residual
    with the native FP64 operator: the same solve converges to the same
    tolerance, with the same iteration count to within a few."""
    dims = (8, 8, 8, 8)
    op, lat = _lat(dims, 1100, kappa=0.1400, mu=0.005)
    tm = lat.tm
    try:
        b = F.odd_spinor(dims, 2100)
        infos = []
        for upd in (0, 1):
            x = to_dev(np.zeros_like(b))
            sp = tm.solve_params(tol=1e-10, sloppy=tm.TM_F16, fp64_updates=upd)
            infos.append(tm.tm_solve_cg(lat.ctx, tm.TM_MDAGM, sp, x, to_dev(b)))
            assert S.rel_residual(op.MdagM, from_dev(x, b.shape), b) <= 1.05e-10
        assert abs(infos[0].iters - infos[1].iters) <= 3
    finally:
        lat.close()


def test_qpqm_and_host_pointers_and_initial_guess():
    dims = (6, 4, 4, 6)
    op, lat = _lat(dims, 1200)
    tm = lat.tm
    try:
        b = F.odd_spinor(dims, 2200)
        x0 = 0.1 * F.odd_spinor(dims, 2201)
        xh = np.ascontiguousarray(x0.copy())           # host buffers
        info = tm.tm_solve_cg(lat.ctx, tm.TM_QPQM, tm.solve_params(tol=1e-11, sloppy=tm.TM_F32), xh,
                              np.ascontiguousarray(b))
        assert S.rel_residual(op.QpQm, xh, b) <= 1.05e-11
        assert info.status == 0
    finally:
        lat.close()


@pytest.mark.parametrize("nf", [1, 2], ids=["light", "heavy"])
def test_converged_initial_guess_returns_fp64_residual(nf):
    """A mixed solve started from a solution: the double-word initial residual
    is below the tolerance, the library confirms it with the FP64 operator and
    returns without iterating; the returned residual is the FP64 one (checked
    against the oracle's)."""
    dims = (6, 4, 4, 6)
    if nf == 1:
        op, lat = _lat(dims, 1250)
        A, b = op.MdagM, F.odd_spinor(dims, 2250)
    else:
        op, lat = _lat(dims, 1251, mubar=0.1246, epsbar=0.1350)
        A, b = op.heavy_sq, F.odd_spinor(dims, 2251, 2)
    tm = lat.tm
    code = tm.TM_MDAGM if nf == 1 else tm.TM_QH_SQ
    try:
        x = to_dev(np.zeros_like(b))
        sp = tm.solve_params(tol=1e-10, sloppy=tm.TM_F16)
        tm.tm_solve_cg(lat.ctx, code, sp, x, to_dev(b))
        xs = from_dev(x, b.shape)
        res = S.rel_residual(A, xs, b)
        assert res <= 1.05e-10
        info = tm.tm_solve_cg(lat.ctx, code, sp, x, to_dev(b))
        assert info.status == 0 and info.iters == 0 and info.reliable_updates == 0
        assert abs(info.true_rel_res - res) <= 1e-3 * res
        assert rel(from_dev(x, b.shape), xs) == 0.0
    finally:
        lat.close()


def test_heavy_cg():
    dims = (4, 4, 4, 8)
    op, lat = _lat(dims, 1300, kappa=0.14, mu=0.0, mubar=0.1246, epsbar=0.135)
    tm = lat.tm
    try:
        b = F.odd_spinor(dims, 2300, 2)
        x = to_dev(np.zeros_like(b))
        tm.tm_solve_cg(lat.ctx, tm.TM_QH_SQ, tm.solve_params(tol=1e-10, sloppy=tm.TM_F32), x, to_dev(b))
        assert S.rel_residual(op.heavy_sq, from_dev(x, b.shape), b) <= 1.05e-10
    finally:
        lat.close()


# (multishift storage, refinement storage); refine 0 = same as the multishift.
# (1, 3) is Sec. 4.2's single-precision MS-CG with double-half refinement.
@pytest.mark.parametrize("sloppy,refine", [(0, 0), (1, 0), (3, 0), (1, 3), (1, 2)],
                         ids=["f64", "f32", "f16", "f32-f16", "f32-bf16"])
def test_multishift_heavy_refined(sloppy, refine):
    dims = (4, 4, 4, 4)
    op, lat = _lat(dims, 1400, kappa=0.14, mu=0.0, mubar=0.1246, epsbar=0.135)
    tm = lat.tm
    try:
        b = F.odd_spinor(dims, 2400, 2)
        shifts = [0.3, 1e-4, 0.02, 1e-3]          # unsorted on purpose
        xs = [to_dev(np.zeros_like(b)) for _ in shifts]
        sp = tm.solve_params(tol=1e-10, sloppy=sloppy, refine=refine)
        infos = tm.tm_solve_multishift(lat.ctx, tm.TM_QH_SQ, shifts, xs, to_dev(b), sp)
        for s, x, inf in zip(shifts, xs, infos):
            A = lambda v, s=s: op.heavy_sq(v) + s * v
            assert S.rel_residual(A, from_dev(x, b.shape), b) <= 1.05e-10
            assert inf.status == 0
    finally:
        lat.close()


def test_multishift_light_matches_oracle_multishift():
    dims = (4, 4, 4, 4)
    op, lat = _lat(dims, 1450)
    tm = lat.tm
    try:
        b = F.odd_spinor(dims, 2450)
        shifts = [1e-3, 0.05, 0.5]
        xs = [to_dev(np.zeros_like(b)) for _ in shifts]
        tm.tm_solve_multishift(lat.ctx, tm.TM_MDAGM, shifts, xs, to_dev(b),
                               tm.solve_params(tol=1e-11, sloppy=tm.TM_F64))
        xo, _ = S.multishift_cg(op.MdagM, b, shifts, tol=1e-12, maxiter=5000)
        for x, r in zip(xs, xo):
            assert rel(from_dev(x, b.shape), r) < 1e-9
    finally:
        lat.close()


def test_power_iteration_vs_dense():
    dims = (2, 2, 2, 4)
    op, lat = _lat(dims, 1500, kappa=0.14, mu=0.0, mubar=0.1246, epsbar=0.135)
    tm = lat.tm
    try:
        vh = op.geo.V // 2
        Qh = S.dense_matrix(lambda v: op.Qhat_heavy(v, +1), vh, (2, 4, 3))
        lam_dense = np.linalg.eigvalsh(Qh @ Qh.conj().T).max()
        lam = tm.tm_power_iteration(lat.ctx, tm.TM_QH_SQ, 2000)
        assert abs(lam - lam_dense) < 1e-6 * lam_dense
    finally:
        lat.close()


def test_batch_uneven_volumes():
    dl = [(4, 4, 4, 4), (6, 4, 4, 6), (4, 4, 4, 8), (8, 6, 4, 10), (4, 4, 4, 4)]
    ops, lats, bs, xs = [], [], [], []
    try:
        for i, d in enumerate(dl):
            op, lat = _lat(d, 3000 + i, kappa=0.14, mu=0.002 + 0.001 * i)
            ops.append(op)
            lats.append(lat)
            b = F.odd_spinor(d, 3100 + i)
            bs.append(b)
            xs.append(to_dev(np.zeros_like(b)))
        tm = lats[0].tm
        for sloppy in (tm.TM_F32, tm.TM_F64, tm.TM_F16):
            for x in xs:
                x.zero_()
            infos = tm.tm_solve_batch([l.ctx for l in lats], tm.TM_MDAGM,
                                      tm.solve_params(tol=1e-10, sloppy=sloppy),
                                      xs, [to_dev(b) for b in bs])
            for op, b, x, inf in zip(ops, bs, xs, infos):
                assert S.rel_residual(op.MdagM, from_dev(x, b.shape), b) <= 1.05e-10
                assert inf.status == 0
    finally:
        for l in lats:
            l.close()


# --- edge cases and failure paths (host-side, no device fault) ---------------
def test_zero_rhs_gives_zero():
    dims = (4, 4, 4, 4)
    op, lat = _lat(dims, 1600)
    tm = lat.tm
    try:
        b = np.zeros((128, 4, 3), complex)
        x = to_dev(F.odd_spinor(dims, 1))
        info = tm.tm_solve_cg(lat.ctx, tm.TM_MDAGM, tm.solve_params(), x, to_dev(b))
        assert np.all(from_dev(x, b.shape) == 0) and info.iters == 0
    finally:
        lat.close()


def test_maxiter_and_nan_and_stale():
    dims = (4, 4, 4, 4)
    op, lat = _lat(dims, 1700)
    tm = lat.tm
    try:
        b = F.odd_spinor(dims, 1701)
        x = to_dev(np.zeros_like(b))
        info = tm.tm_solve_cg(lat.ctx, tm.TM_MDAGM, tm.solve_params(maxiter=3, chunk=2), x, to_dev(b),
                              check=False)
        assert info.status == tm.TM_ERR_NOT_CONVERGED
        bn = b.copy()
        bn[3, 1, 2] = np.nan
        x.zero_()
        info = tm.tm_solve_cg(lat.ctx, tm.TM_MDAGM, tm.solve_params(), x, to_dev(bn), check=False)
        assert info.status == tm.TM_ERR_BREAKDOWN
        # a new gauge field makes the clover term stale (Sec. 3 cascade)
        tm.tm_gauge_load(lat.ctx, np.ascontiguousarray(F.gauge_field(dims, 1702)), 2.0)
        assert tm.tm_gauge_id(lat.ctx) == 2.0
        with pytest.raises(tm.TMError) as e:
            lat.apply(tm.TM_QHAT_PLUS, 0, b)
        assert e.value.status == tm.TM_ERR_STALE
        tm.tm_clover_compute(lat.ctx, 0.1394, CSW, mu=0.01)
        lat.apply(tm.TM_QHAT_PLUS, 0, b)
    finally:
        lat.close()


def test_solvers_with_staged_kernels():
    """Mixed CG, multishift and batch with the staged stencil variant."""
    dims = (8, 8, 8, 8)
    op, lat = _lat(dims, 1800, kappa=0.14, mu=0.004, mubar=0.1246, epsbar=0.135)
    tm = lat.tm
    try:
        for prec in (tm.TM_F32, tm.TM_F16):
            for nf in (1, 2):
                tm.tm_set_tuning(lat.ctx, prec, nf, 1, 1)
        b = F.odd_spinor(dims, 1801)
        x = to_dev(np.zeros_like(b))
        tm.tm_solve_cg(lat.ctx, tm.TM_MDAGM, tm.solve_params(tol=1e-10, sloppy=tm.TM_F16), x, to_dev(b))
        assert S.rel_residual(op.MdagM, from_dev(x, b.shape), b) <= 1.05e-10
        b2 = F.odd_spinor(dims, 1802, 2)
        shifts = [1e-3, 0.1]
        xs = [to_dev(np.zeros_like(b2)) for _ in shifts]
        tm.tm_solve_multishift(lat.ctx, tm.TM_QH_SQ, shifts, xs, to_dev(b2), tm.solve_params(sloppy=tm.TM_F32))
        for s, xx in zip(shifts, xs):
            assert S.rel_residual(lambda v, s=s: op.heavy_sq(v) + s * v, from_dev(xx, b2.shape), b2) <= 1.05e-10
        x.zero_()
        tm.tm_solve_batch([lat.ctx], tm.TM_MDAGM, tm.solve_params(sloppy=tm.TM_F16), [x], [to_dev(b)])
        assert S.rel_residual(op.MdagM, from_dev(x, b.shape), b) <= 1.05e-10
    finally:
        lat.close()


def test_cg_on_W_hat_normal_operator():
    dims = (6, 4, 4, 6)
    u = F.gauge_field(dims, 1900)
    op = D.TwistedMassClover(u, dims, 0.14, CSW, mu=0.004)
    lat = Lat(u, dims, 0.14, CSW, mu=0.004, rho=0.1)
    tm = lat.tm
    try:
        b = F.odd_spinor(dims, 1901)
        x = to_dev(np.zeros_like(b))
        tm.tm_solve_cg(lat.ctx, tm.TM_WHAT_SQ, tm.solve_params(tol=1e-10, sloppy=tm.TM_F16), x, to_dev(b))
        A = lambda v: op.What(op.What(v, 0.1, +1), 0.1, -1)
        assert S.rel_residual(A, from_dev(x, b.shape), b) <= 1.05e-10
    finally:
        lat.close()


def test_pinned_host_fields_are_stream_ordered_and_overlap():
    """Imports and exports with pinned host buffers on their own streams, the
    operator on a third, several steps in flight (the bench's end-to-end loop):
    every result equals the synchronous device-pointer path."""
    import torch
    dims = (4, 4, 4, 8)
    op, lat = _lat(dims, 1700)
    tm = lat.tm
    try:
        rhs = [F.odd_spinor(dims, 2700 + k) for k in range(5)]
        ref = []
        for b in rhs:
            fi = lat.native(tm.TM_F32, 1)
            fo = lat.native(tm.TM_F32, 1)
            tm.tm_field_import(lat.ctx, tm.TM_F32, 1, fi, to_dev(b))
            tm.tm_apply_Mhat(lat.ctx, tm.TM_MDAGM, tm.TM_F32, fo, fi)
            o = to_dev(np.zeros_like(b))
            tm.tm_field_export(lat.ctx, tm.TM_F32, 1, o, fo)
            torch.cuda.synchronize()
            ref.append(from_dev(o, b.shape))
        hin = [torch.from_numpy(b.view(np.float64).reshape(-1).copy()).pin_memory() for b in rhs]
        hout = [torch.zeros_like(h).pin_memory() for h in hin]
        fins = [lat.native(tm.TM_F32, 1) for _ in range(2)]
        fouts = [lat.native(tm.TM_F32, 1) for _ in range(2)]
        s_in, s_op, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_op = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        for k in range(len(rhs)):
            i = k % 2
            if k >= 2:
                s_in.wait_event(ev_op[i])
            tm.tm_field_import(lat.ctx, tm.TM_F32, 1, fins[i], hin[k], stream=s_in)
            ev_in[i].record(s_in)
            s_op.wait_event(ev_in[i])
            if k >= 2:
                s_op.wait_event(ev_out[i])
            tm.tm_apply_Mhat(lat.ctx, tm.TM_MDAGM, tm.TM_F32, fouts[i], fins[i], stream=s_op)
            ev_op[i].record(s_op)
            s_out.wait_event(ev_op[i])
            tm.tm_field_export(lat.ctx, tm.TM_F32, 1, hout[k], fouts[i], stream=s_out)
            ev_out[i].record(s_out)
        torch.cuda.synchronize()
        for k, b in enumerate(rhs):
            got = hout[k].numpy().view(np.complex128).reshape(b.shape)
            assert np.array_equal(got, ref[k])
    finally:
        lat.close()
