"""Parity of the CUDA operators (clover term, Q_hat_pm of eq:hQpm, Q_hat_h of
eq:hQh and their normal products) against the FP64 CPU oracle, element by
element, in every storage precision."""
import numpy as np
import pytest

from oracle import dirac as D
from synth import fields as F
from tests.gpu_util import DW_TOL, Lat, rel, tol

pytestmark = pytest.mark.gpu

KAPPA, CSW, MU, MUBAR, EPSBAR = 0.1394, 1.69, 0.01, 0.1246, 0.1350
# lattices spanning several 128-site tiles with ragged tails, plus the minimum 2^4
DIMS = [(4, 4, 4, 4), (6, 4, 4, 6), (2, 2, 2, 2), (8, 6, 4, 10)]


@pytest.fixture(scope="module", params=DIMS, ids=lambda d: "x".join(map(str, d)))
def setup(request):
    dims = request.param
    u = F.gauge_field(dims, 1000 + sum(dims))
    op = D.TwistedMassClover(u, dims, KAPPA, CSW, mu=MU, mubar=MUBAR, epsbar=EPSBAR)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU, mubar=MUBAR, epsbar=EPSBAR)
    yield dims, op, lat
    lat.close()


def test_clover_term_fp64(setup):
    import torch
    dims, op, lat = setup
    vh = lat.vh
    for par, sites in ((0, op.geo.even), (1, op.geo.odd)):
        out = torch.empty(vh * 2 * 36 * 2, dtype=torch.float64, device="cuda:0")
        lat.tm.tm_clover_export(lat.ctx, par, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.complex128).reshape(vh, 2, 6, 6)
        A = op.A[sites]
        ref = np.stack([A[:, :6, :6], A[:, 6:, 6:]], axis=1)
        assert rel(got, ref) < 1e-14


@pytest.mark.parametrize("prec", [0, 1, 3, 2], ids=["f64", "f32", "f16", "bf16"])
def test_light_schur_operators(setup, prec):
    dims, op, lat = setup
    tm = lat.tm
    psi = F.odd_spinor(dims, 7)
    for code, ref, n in ((tm.TM_QHAT_PLUS, op.Qhat(psi, +1), 1), (tm.TM_QHAT_MINUS, op.Qhat(psi, -1), 1),
                         (tm.TM_MDAGM, op.MdagM(psi), 2), (tm.TM_QPQM, op.QpQm(psi), 2)):
        got = lat.apply(code, prec, psi)
        assert rel(got, ref) < tol(prec, n), (code, rel(got, ref))


@pytest.mark.parametrize("prec", [0, 1, 3, 2], ids=["f64", "f32", "f16", "bf16"])
def test_heavy_schur_operators(setup, prec):
    dims, op, lat = setup
    tm = lat.tm
    psi = F.odd_spinor(dims, 8, 2)
    for code, ref, n in ((tm.TM_QH, op.Qhat_heavy(psi, +1), 1), (tm.TM_QH_DAG, op.Qhat_heavy(psi, -1), 1),
                         (tm.TM_QH_SQ, op.heavy_sq(psi), 2)):
        got = lat.apply(code, prec, psi)
        assert rel(got, ref) < tol(prec, n), (code, rel(got, ref))


def test_double_word_operators(setup):
    """tm_apply_Mhat_dw (the reliable updates' operator) against the oracle and
    against the native FP64 operator, light and heavy, single and normal."""
    dims, op, lat = setup
    tm = lat.tm
    psi = F.odd_spinor(dims, 7)
    psih = F.odd_spinor(dims, 8, 2)
    for code, ref, x, n in ((tm.TM_QHAT_PLUS, op.Qhat(psi, +1), psi, 1), (tm.TM_QHAT_MINUS, op.Qhat(psi, -1), psi, 1),
                            (tm.TM_MDAGM, op.MdagM(psi), psi, 2), (tm.TM_QPQM, op.QpQm(psi), psi, 2),
                            (tm.TM_QH, op.Qhat_heavy(psih, +1), psih, 1),
                            (tm.TM_QH_DAG, op.Qhat_heavy(psih, -1), psih, 1),
                            (tm.TM_QH_SQ, op.heavy_sq(psih), psih, 2)):
        got = lat.apply_dw(code, x)
        assert rel(got, ref) < n * DW_TOL, (code, rel(got, ref))
        assert rel(got, lat.apply(code, 0, x)) < n * DW_TOL, code


def test_double_word_copies_follow_the_gauge_field():
    """The double-word links and clover blocks are remade after a new gauge field
    and clover term."""
    dims = (4, 4, 4, 6)
    u1 = F.gauge_field(dims, 31)
    u2 = F.gauge_field(dims, 32)
    lat = Lat(u1, dims, KAPPA, CSW, mu=MU)
    try:
        psi = F.odd_spinor(dims, 33)
        op1 = D.TwistedMassClover(u1, dims, KAPPA, CSW, mu=MU)
        assert rel(lat.apply_dw(lat.tm.TM_MDAGM, psi), op1.MdagM(psi)) < 2 * DW_TOL
        lat.tm.tm_gauge_load(lat.ctx, np.ascontiguousarray(u2), 2.0)
        lat.tm.tm_clover_compute(lat.ctx, KAPPA, CSW, mu=2 * MU)
        op2 = D.TwistedMassClover(u2, dims, KAPPA, CSW, mu=2 * MU)
        assert rel(lat.apply_dw(lat.tm.TM_MDAGM, psi), op2.MdagM(psi)) < 2 * DW_TOL
    finally:
        lat.close()


def test_host_pointers_for_native_fields_are_rejected():
    """Native fields must be device memory: every entry point that hands one to a
    kernel returns TM_ERR_ARG for a host pointer before launching anything."""
    import torch
    dims = (4, 4, 4, 4)
    lat = Lat(F.gauge_field(dims, 41), dims, KAPPA, CSW, mu=MU)
    tm = lat.tm
    try:
        nb = tm.tm_field_bytes(lat.ctx, 0, 1)
        dev = lat.native(0, 1)
        host = np.zeros(nb // 8 + 2, dtype=np.float64)   # 16-byte aligned numpy buffer
        hp = host.ctypes.data
        hp += (-hp) % 16
        dp = dev.data_ptr()
        canon = torch.zeros(lat.vh * 24, dtype=torch.float64, device="cuda:0")
        res = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        calls = [
            ("tm_apply_Mhat", lambda: tm.lib.tm_apply_Mhat(lat.ctx, tm.TM_MDAGM, 0, hp, dp, None)),
            ("tm_apply_Mhat", lambda: tm.lib.tm_apply_Mhat(lat.ctx, tm.TM_MDAGM, 0, dp, hp, None)),
            ("tm_apply_Mhat_dw", lambda: tm.lib.tm_apply_Mhat_dw(lat.ctx, tm.TM_MDAGM, hp, dp, None)),
            ("tm_apply_even", lambda: tm.lib.tm_apply_even(lat.ctx, tm.TM_QHAT_PLUS, 0, hp, dp, None)),
            ("tm_field_import", lambda: tm.lib.tm_field_import(lat.ctx, 0, 1, hp, canon.data_ptr(), None)),
            ("tm_field_export", lambda: tm.lib.tm_field_export(lat.ctx, 0, 1, canon.data_ptr(), hp, None)),
            ("tm_field_norm2", lambda: tm.lib.tm_field_norm2(lat.ctx, 0, 1, hp, res.data_ptr(), None)),
        ]
        for name, call in calls:
            assert call() == tm.TM_ERR_ARG, name
            assert "device pointer" in tm.tm_last_error(), name
        torch.cuda.synchronize()   # nothing was launched with the host address
    finally:
        lat.close()


def test_periodic_time_boundary():
    dims = (4, 4, 2, 6)
    u = F.gauge_field(dims, 31)
    op = D.TwistedMassClover(u, dims, KAPPA, CSW, mu=MU, bc_t=+1)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU, bc_t=+1)
    try:
        psi = F.odd_spinor(dims, 32)
        assert rel(lat.apply(lat.tm.TM_QHAT_PLUS, 0, psi), op.Qhat(psi, +1)) < 1e-13
        assert rel(lat.apply_dw(lat.tm.TM_MDAGM, psi), op.MdagM(psi)) < 2 * DW_TOL
    finally:
        lat.close()


def _two_hop_odd(geo, odd_idx):
    """Odd-list indices of the odd sites within two hops (odd -> even -> odd) of
    the given odd sites: the support of Q_hat at those sites."""
    S = geo.odd[np.asarray(odd_idx)]
    e = np.unique(np.concatenate([geo.fwd[m][S] for m in range(4)] + [geo.bwd[m][S] for m in range(4)]))
    o = np.unique(np.concatenate([geo.fwd[m][e] for m in range(4)] + [geo.bwd[m][e] for m in range(4)]))
    return o // 2


@pytest.fixture(scope="module")
def full32():
    """32^3x64, the mixed-precision CG workload, and 67 sampled odd sites."""
    dims = (32, 32, 32, 64)
    u = F.gauge_field(dims, 1001)
    op = D.TwistedMassClover(u, dims, 0.1400, CSW, mu=0.0015)
    lat = Lat(u, dims, 0.1400, CSW, mu=0.0015)
    psi = F.odd_spinor(dims, 2001)
    rng = np.random.default_rng(5)
    s = np.unique(np.concatenate([[0, 1, lat.vh - 1], rng.integers(0, lat.vh, 64)]))
    # M_hat^dag M_hat = Q_hat_- Q_hat_+ at s needs Q_hat_+ psi on the odd sites
    # within two hops of s; the oracle evaluates it there only
    n2 = _two_hop_odd(op.geo, s)
    mid = np.zeros_like(psi)
    mid[n2] = op.Qhat_at(psi, n2, +1)
    refs = {"qp": op.Qhat_at(psi, s, +1), "mdagm": op.Qhat_at(mid, s, -1)}
    yield lat, psi, s, refs
    lat.close()


@pytest.mark.parametrize("prec", [0, 1, 3, 2], ids=["f64", "f32", "f16", "bf16"])
def test_full_size_sampled_32x64(full32, prec):
    """32^3x64 in the launch configuration the benchmark uses (autotuned
    variant, every storage precision): Q_hat_+ and M_hat^dag M_hat checked at
    sampled odd sites, including the first and the last."""
    lat, psi, s, refs = full32
    tm = lat.tm
    if prec != 0:
        tm.tm_autotune(lat.ctx, prec, 1)
    got = lat.apply(tm.TM_QHAT_PLUS, prec, psi)[s]
    assert rel(got, refs["qp"]) < tol(prec), (prec, rel(got, refs["qp"]))
    got = lat.apply(tm.TM_MDAGM, prec, psi)[s]
    assert rel(got, refs["mdagm"]) < tol(prec, 2), (prec, rel(got, refs["mdagm"]))


@pytest.fixture(scope="module")
def heavy24():
    """24^3x48, the heavy-doublet multishift workload (mubar 0.1246, epsbar 0.1350),
    and 40 sampled odd sites."""
    dims = (24, 24, 24, 48)
    u = F.gauge_field(dims, 1002)
    op = D.TwistedMassClover(u, dims, 0.1400, CSW, mubar=0.1246, epsbar=0.1350)
    lat = Lat(u, dims, 0.1400, CSW, mubar=0.1246, epsbar=0.1350)
    psi = F.odd_spinor(dims, 2002, 2)
    rng = np.random.default_rng(6)
    s = np.unique(np.concatenate([[0, lat.vh - 1], rng.integers(0, lat.vh, 38)]))
    n2 = _two_hop_odd(op.geo, s)
    mid = np.zeros_like(psi)
    mid[n2] = op.Qhat_at(psi, n2, -1, heavy=True)
    refs = {"qh": op.Qhat_at(psi, s, +1, heavy=True), "qhsq": op.Qhat_at(mid, s, +1, heavy=True)}
    yield lat, psi, s, refs
    lat.close()


@pytest.mark.parametrize("prec", [0, 1, 3, 2], ids=["f64", "f32", "f16", "bf16"])
def test_full_size_sampled_heavy_24x48(heavy24, prec):
    """The heavy doublet at the multishift workload's size, in the variant the
    autotuner picks (the even pass splits the flavours over thread pairs):
    Q_hat_h and Q_hat_h Q_hat_h^dag at sampled odd sites."""
    lat, psi, s, refs = heavy24
    tm = lat.tm
    if prec != 0:
        tm.tm_autotune(lat.ctx, prec, 2)
    got = lat.apply(tm.TM_QH, prec, psi)[s]
    assert rel(got, refs["qh"]) < tol(prec), (prec, rel(got, refs["qh"]))
    got = lat.apply(tm.TM_QH_SQ, prec, psi)[s]
    assert rel(got, refs["qhsq"]) < tol(prec, 2), (prec, rel(got, refs["qhsq"]))


def test_full_size_sampled_48x96_f16():
    """48^3x96, the learned-preconditioner and multigrid workload (kappa
    0.1394265, mu 0.00072), in FP16 storage and FP64: Q_hat_+ at sampled odd
    sites, including the last."""
    dims = (48, 48, 48, 96)
    u = F.gauge_field(dims, 1004)
    op = D.TwistedMassClover(u, dims, 0.1394265, CSW, mu=0.00072)
    lat = Lat(u, dims, 0.1394265, CSW, mu=0.00072)
    try:
        psi = F.odd_spinor(dims, 2004)
        rng = np.random.default_rng(7)
        s = np.unique(np.concatenate([[0, lat.vh - 1], rng.integers(0, lat.vh, 30)]))
        ref = op.Qhat_at(psi, s, +1)
        lat.tm.tm_autotune(lat.ctx, lat.tm.TM_F16, 1)
        for prec in (0, 3):
            got = lat.apply(lat.tm.TM_QHAT_PLUS, prec, psi)[s]
            assert rel(got, ref) < tol(prec), (prec, rel(got, ref))
    finally:
        lat.close()


@pytest.mark.parametrize("prec", [1, 3, 2], ids=["f32", "f16", "bf16"])
def test_staged_variant_matches_oracle(setup, prec):
    """The shared-memory staged stencil kernels give the oracle's operator too
    (light and heavy, both passes forced to the staged variant)."""
    dims, op, lat = setup
    tm = lat.tm
    psi = F.odd_spinor(dims, 9)
    psi2 = F.odd_spinor(dims, 10, 2)
    for ev, od in ((1, 1), (1, 0), (0, 1)):
        tm.tm_set_tuning(lat.ctx, prec, 1, ev, od)
        tm.tm_set_tuning(lat.ctx, prec, 2, ev, od)
        assert rel(lat.apply(tm.TM_QHAT_PLUS, prec, psi), op.Qhat(psi, +1)) < tol(prec)
        assert rel(lat.apply(tm.TM_MDAGM, prec, psi), op.MdagM(psi)) < tol(prec, 2)
        assert rel(lat.apply(tm.TM_QH_DAG, prec, psi2), op.Qhat_heavy(psi2, -1)) < tol(prec)
    tm.tm_set_tuning(lat.ctx, prec, 1, 0, 0)
    tm.tm_set_tuning(lat.ctx, prec, 2, 0, 0)


def test_autotune_choice_is_kept():
    dims = (8, 8, 4, 8)
    u = F.gauge_field(dims, 61)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU)
    try:
        tm = lat.tm
        choice = tm.tm_autotune(lat.ctx, tm.TM_F16, 1)
        assert tm.tm_get_tuning(lat.ctx, tm.TM_F16, 1) == choice
        assert tm.tm_autotune(lat.ctx, tm.TM_F64, 1) == (0, 0)
        with pytest.raises(tm.TMError):
            tm.tm_set_tuning(lat.ctx, tm.TM_F64, 1, 1, 1)
    finally:
        lat.close()


@pytest.mark.parametrize("prec", [0, 1, 3], ids=["f64", "f32", "f16"])
def test_mass_preconditioned_W_hat(prec):
    """W_hat_pm(rho) = Q_hat_pm pm i rho (eq:hWpm) and W_hat_- W_hat_+; changing rho
    leaves the clover term untouched (it is rho-independent, Sec. 2)."""
    dims = (6, 4, 4, 6)
    u = F.gauge_field(dims, 71)
    op = D.TwistedMassClover(u, dims, KAPPA, CSW, mu=MU)
    lat = Lat(u, dims, KAPPA, CSW, mu=MU)
    try:
        tm = lat.tm
        psi = F.odd_spinor(dims, 72)
        for rho in (0.05, 0.3):
            tm.tm_clover_compute(lat.ctx, KAPPA, CSW, mu=MU, rho=rho)
            wp = op.What(psi, rho, +1)
            wm = op.What(psi, rho, -1)
            wsq = op.What(op.What(psi, rho, +1), rho, -1)
            assert rel(lat.apply(tm.TM_WHAT_PLUS, prec, psi), wp) < tol(prec)
            assert rel(lat.apply(tm.TM_WHAT_MINUS, prec, psi), wm) < tol(prec)
            assert rel(lat.apply(tm.TM_WHAT_SQ, prec, psi), wsq) < tol(prec, 2)
            if prec == 0:   # and the double-word form of the reliable updates
                assert rel(lat.apply_dw(tm.TM_WHAT_PLUS, psi), wp) < DW_TOL
                assert rel(lat.apply_dw(tm.TM_WHAT_MINUS, psi), wm) < DW_TOL
                assert rel(lat.apply_dw(tm.TM_WHAT_SQ, psi), wsq) < 2 * DW_TOL
    finally:
        lat.close()
