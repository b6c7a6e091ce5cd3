"""Parity of the GPU two-level multigrid (the multigrid-preconditioned GCR of
Sec. 4.1) with the FP64 oracle of oracle/multigrid.py, step by step: the full
operator, the smoothed near-null vectors, the Gram-Schmidt prolongator and its
adjoint, the Galerkin coarse operator, the preconditioner, and the GCR solves.

Both sides start the setup from the same seeded random fields (the method draws
them; they are inputs here).  FP64 mode is compared element by element at
1e-13 (operator) to 1e-9 (quantities after iterations); FP32 mode against the
oracle built from the GPU's own near-null vectors at FP32 tolerances, and every
solve by the oracle's FP64 residual of the returned solution.
"""
import numpy as np
import pytest

from oracle import dirac as D
from oracle import multigrid as MG
from synth import fields as F
from tests.gpu_util import rel, to_dev, from_dev

pytestmark = pytest.mark.gpu

KAPPA, CSW, MU = 0.1394, 1.69, 0.01


def _op(dims, seed, bc_t=-1, mu=MU):
    u = F.gauge_field(dims, seed)
    return u, D.TwistedMassClover(u, dims, KAPPA, CSW, mu=mu, bc_t=bc_t)


def _ctx(tm, u, dims, bc_t=-1, mu=MU):
    ctx = tm.tm_create(dims, 0)
    tm.tm_gauge_load(ctx, np.ascontiguousarray(u), 1.0)
    tm.tm_clover_compute(ctx, KAPPA, CSW, mu=mu, bc_t=bc_t)
    return ctx


def _full(dims, seed):
    return F.spinor((int(np.prod(dims)), 4, 3), seed)


@pytest.mark.parametrize("dims,bc_t", [((4, 4, 4, 4), -1), ((6, 4, 4, 6), -1), ((8, 6, 4, 10), 1)],
                         ids=["4x4x4x4", "6x4x4x6", "8x6x4x10-periodic"])
def test_full_operator(dims, bc_t):
    import torch
    from paper_2212_06635_gb300 import tm
    u, op = _op(dims, 1900 + sum(dims), bc_t)
    ctx = _ctx(tm, u, dims, bc_t)
    try:
        psi = _full(dims, 11)
        src = to_dev(psi)
        out = torch.empty_like(src)
        for sign in (1, -1):
            ref = op.M(psi, sign)
            for prec, tol in ((tm.TM_F64, 1e-13), (tm.TM_F32, 1e-6)):
                tm.tm_apply_full(ctx, sign, prec, out, src)
                torch.cuda.synchronize()
                assert rel(from_dev(out, psi.shape), ref) < tol, (sign, prec)
    finally:
        tm.tm_destroy(ctx)


class _Pair:
    """A GPU multigrid and the oracle's, set up from the same starting fields."""

    def __init__(self, dims, block, nvec, setup_steps=10, smooth_steps=2, sign=1, seed=1931, prec=0,
                 coarse_tol=1e-13, oracle_from_gpu_vectors=False):
        import torch
        from paper_2212_06635_gb300 import tm
        self.tm = tm
        self.dims = dims
        self.u, self.op = _op(dims, seed)
        self.ctx = _ctx(tm, self.u, dims)
        V = int(np.prod(dims))
        self.V = V
        init = np.stack([_full(dims, seed + 10 + j) for j in range(nvec)])
        self.mg = tm.tm_mg_create(self.ctx, tm.mg_params(block, nvec, setup_steps, smooth_steps, sign, prec,
                                                         coarse_tol, 5000, 16))
        tm.tm_mg_setup(self.mg, to_dev(init))
        vec = torch.empty(nvec * V * 24, dtype=torch.float64, device="cuda")
        tm.tm_mg_vectors(self.mg, vec)
        torch.cuda.synchronize()
        self.gpu_vectors = from_dev(vec, (nvec, V, 4, 3))
        if oracle_from_gpu_vectors:
            self.ref = MG.TwoLevelMG(self.op, block, nvec, smooth_steps=smooth_steps, sign=sign,
                                     vectors=list(self.gpu_vectors))
        else:
            self.ref = MG.TwoLevelMG(self.op, block, nvec, setup_steps=setup_steps, smooth_steps=smooth_steps,
                                     sign=sign, init=init)
        self.nc = tm.tm_mg_coarse_size(self.mg)
        assert self.nc == self.ref.ncoarse

    def close(self):
        self.tm.tm_mg_destroy(self.mg)
        self.tm.tm_destroy(self.ctx)


@pytest.fixture(scope="module")
def pair64():
    p = _Pair((4, 4, 4, 8), (2, 2, 2, 2), 4)
    yield p
    p.close()


def test_near_null_vectors_fp64(pair64):
    p = pair64
    for j in range(len(p.ref.vectors)):
        assert rel(p.gpu_vectors[j], p.ref.vectors[j]) < 1e-11, j
        assert abs(np.linalg.norm(p.gpu_vectors[j]) - 1.0) < 1e-13


def test_prolong_restrict_fp64(pair64):
    import torch
    p, tm = pair64, pair64.tm
    gen = np.random.default_rng(3)
    uc = gen.standard_normal(p.nc) + 1j * gen.standard_normal(p.nc)
    fine = torch.empty(p.V * 24, dtype=torch.float64, device="cuda")
    tm.tm_mg_prolong(p.mg, fine, to_dev(uc))
    torch.cuda.synchronize()
    pu = from_dev(fine, (p.V, 4, 3))
    assert rel(pu, p.ref.prolong(uc)) < 1e-11
    v = _full(p.dims, 41)
    cout = torch.empty(2 * p.nc, dtype=torch.float64, device="cuda")
    tm.tm_mg_restrict(p.mg, cout, to_dev(v))
    torch.cuda.synchronize()
    assert rel(from_dev(cout, (p.nc,)), p.ref.restrict(v)) < 1e-11
    # P^+ P = 1 on the GPU side alone
    tm.tm_mg_restrict(p.mg, cout, fine)
    torch.cuda.synchronize()
    assert rel(from_dev(cout, (p.nc,)), uc) < 1e-13


def test_coarse_operator_fp64(pair64):
    import torch
    p, tm = pair64, pair64.tm
    Mc = p.ref.coarse_matrix()
    gen = np.random.default_rng(4)
    out = torch.empty(2 * p.nc, dtype=torch.float64, device="cuda")
    for _ in range(2):
        uc = gen.standard_normal(p.nc) + 1j * gen.standard_normal(p.nc)
        tm.tm_mg_coarse_apply(p.mg, out, to_dev(uc))
        torch.cuda.synchronize()
        assert rel(from_dev(out, (p.nc,)), Mc @ uc) < 1e-11
    # every column: the coarse operator itself, element by element
    E = np.eye(p.nc)
    cols = []
    for j in range(p.nc):
        tm.tm_mg_coarse_apply(p.mg, out, to_dev(E[j].astype(np.complex128)))
        cols.append(from_dev(out, (p.nc,)).copy())
    torch.cuda.synchronize()
    assert np.max(np.abs(np.stack(cols, axis=1) - Mc)) < 1e-12 * np.max(np.abs(Mc))


def test_preconditioner_fp64(pair64):
    import torch
    p, tm = pair64, pair64.tm
    r = _full(p.dims, 51)
    z = torch.empty(p.V * 24, dtype=torch.float64, device="cuda")
    its = tm.tm_mg_precondition(p.mg, z, to_dev(r))
    assert its > 0
    assert rel(from_dev(z, r.shape), p.ref.precondition(r)) < 1e-9


def test_mg_gcr_solve_fp64(pair64):
    import torch
    p, tm = pair64, pair64.tm
    b = _full(p.dims, 61)
    x = torch.zeros(p.V * 24, dtype=torch.float64, device="cuda")
    info = tm.tm_solve_gcr(p.ctx, 1, p.mg, tm.solve_params(tol=1e-10, maxiter=500, chunk=8), x, to_dev(b))
    xs = from_dev(x, b.shape)
    res = np.linalg.norm(b - p.op.M(xs)) / np.linalg.norm(b)
    assert res <= 1.05e-10, res
    assert info.true_rel_res <= 1e-10
    xr, itr = MG.gcr(p.ref.apply, b, p.ref.precondition, tol=1e-10, restart=8)
    # both solutions within the residual bound of each other (condition number of M here < 1e3)
    assert rel(xs, xr) < 1e-7
    assert abs(info.iters - itr) <= 3, (info.iters, itr)


@pytest.mark.parametrize("dims,block,nvec", [((4, 4, 4, 8), (4, 2, 2, 2), 6), ((4, 2, 2, 4), (2, 2, 2, 4), 8),
                                             ((2, 2, 2, 2), (1, 1, 1, 1), 6)],
                         ids=["nb1-in-x", "Vb32-nv8", "one-site-aggregates"])
def test_block_layouts_fp64(dims, block, nvec):
    """Aggregates spanning a whole extent (one block in that direction, hops
    wrapping into the same block), 2 blocks in a direction (forward and backward
    neighbour the same block), and one-site aggregates with nvec = 6 (P unitary:
    the coarse operator is M itself in another basis)."""
    import torch
    p = _Pair(dims, block, nvec, setup_steps=6, seed=1941 + sum(dims))
    try:
        tm = p.tm
        Mc = p.ref.coarse_matrix()
        gen = np.random.default_rng(5)
        uc = gen.standard_normal(p.nc) + 1j * gen.standard_normal(p.nc)
        out = torch.empty(2 * p.nc, dtype=torch.float64, device="cuda")
        tm.tm_mg_coarse_apply(p.mg, out, to_dev(uc))
        torch.cuda.synchronize()
        assert rel(from_dev(out, (p.nc,)), Mc @ uc) < 1e-10
        fine = torch.empty(p.V * 24, dtype=torch.float64, device="cuda")
        tm.tm_mg_prolong(p.mg, fine, to_dev(uc))
        torch.cuda.synchronize()
        assert rel(from_dev(fine, (p.V, 4, 3)), p.ref.prolong(uc)) < 1e-10
        if block == (1, 1, 1, 1):
            # exact coarse space: the preconditioner is M^-1 itself
            b = _full(dims, 71)
            x = torch.zeros(p.V * 24, dtype=torch.float64, device="cuda")
            info = tm.tm_solve_gcr(p.ctx, 1, p.mg, tm.solve_params(tol=1e-12, maxiter=50, chunk=8), x, to_dev(b))
            assert info.iters <= 2, info.iters
            assert np.linalg.norm(b - p.op.M(from_dev(x, b.shape))) <= 1.05e-12 * np.linalg.norm(b)
    finally:
        p.close()


def test_sign_minus_and_gamma5_hermiticity_fp64():
    """The multigrid of M(-mu): its coarse operator against the oracle's, and the
    coarse gamma_5-hermiticity M_c(mu)^+ = G5 M_c(-mu) G5 between the two GPU
    hierarchies built from the same vectors' setup."""
    import torch
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    pp = _Pair(dims, block, 4, setup_steps=0, sign=1, seed=1951)
    pm = _Pair(dims, block, 4, setup_steps=0, sign=-1, seed=1951)
    try:
        tm = pp.tm
        nc = pp.nc
        out = torch.empty(2 * nc, dtype=torch.float64, device="cuda")

        def dense(mg):
            cols = []
            for j in range(nc):
                e = np.zeros(nc, dtype=np.complex128)
                e[j] = 1.0
                tm.tm_mg_coarse_apply(mg, out, to_dev(e))
                cols.append(from_dev(out, (nc,)).copy())
            torch.cuda.synchronize()
            return np.stack(cols, axis=1)

        Mp, Mm = dense(pp.mg), dense(pm.mg)
        assert np.max(np.abs(Mm - pm.ref.coarse_matrix())) < 1e-12 * np.max(np.abs(Mm))
        g = pp.ref.coarse_gamma5()
        assert np.max(np.abs(Mp.conj().T - g[:, None] * Mm * g[None, :])) < 1e-12 * np.max(np.abs(Mp))
    finally:
        pp.close()
        pm.close()


def test_fp32_multigrid_and_gcr_solves():
    """FP32 mode: the coarse operator against the oracle built from the GPU's own
    (FP32-smoothed) vectors, and GCR to FP64 true residual 1e-10 with the FP32
    multigrid, plain FP32 GCR and plain FP64 GCR; the multigrid cuts the
    iteration count (the oracle's gain test, here on the GPU)."""
    import torch
    dims = (8, 8, 8, 8)
    p = _Pair(dims, (4, 4, 4, 4), 8, setup_steps=20, smooth_steps=4, prec=1, coarse_tol=0.05,
              oracle_from_gpu_vectors=True, seed=1961)
    try:
        tm = p.tm
        gen = np.random.default_rng(6)
        uc = gen.standard_normal(p.nc) + 1j * gen.standard_normal(p.nc)
        out = torch.empty(2 * p.nc, dtype=torch.float64, device="cuda")
        tm.tm_mg_coarse_apply(p.mg, out, to_dev(uc))
        torch.cuda.synchronize()
        assert rel(from_dev(out, (p.nc,)), p.ref.coarse_matrix() @ uc) < 1e-5
        b = _full(dims, 81)
        bd = to_dev(b)
        its = {}
        for name, mg, sl in (("mg32", p.mg, tm.TM_F32), ("gcr32", None, tm.TM_F32), ("gcr64", None, tm.TM_F64)):
            x = torch.zeros(p.V * 24, dtype=torch.float64, device="cuda")
            info = tm.tm_solve_gcr(p.ctx, 1, mg, tm.solve_params(tol=1e-10, maxiter=5000, sloppy=sl, chunk=8), x, bd)
            res = np.linalg.norm(b - p.op.M(from_dev(x, b.shape))) / np.linalg.norm(b)
            assert res <= 1.05e-10, (name, res)
            its[name] = info.iters
        assert its["mg32"] * 3 < its["gcr32"], its
    finally:
        p.close()


def test_fp32_preconditioner_and_minus_sign_solve():
    """FP32 hierarchy of M(-mu): the preconditioner against the oracle's built
    from the GPU's own (FP32-smoothed) vectors with an essentially exact coarse
    solve (FP32 tolerance), and the preconditioned GCR solve of M(-mu) x = b to
    an oracle residual of 1e-10."""
    import torch
    dims = (4, 4, 4, 8)
    p = _Pair(dims, (2, 2, 2, 2), 6, setup_steps=10, smooth_steps=3, sign=-1, prec=1, coarse_tol=1e-7,
              oracle_from_gpu_vectors=True, seed=1981)
    try:
        tm = p.tm
        r = _full(dims, 82)
        z = torch.empty(p.V * 24, dtype=torch.float64, device="cuda")
        tm.tm_mg_precondition(p.mg, z, to_dev(r))
        assert rel(from_dev(z, r.shape), p.ref.precondition(r)) < 2e-5
        b = _full(dims, 83)
        x = torch.zeros(p.V * 24, dtype=torch.float64, device="cuda")
        info = tm.tm_solve_gcr(p.ctx, -1, p.mg, tm.solve_params(tol=1e-10, maxiter=2000, sloppy=tm.TM_F32, chunk=8),
                               x, to_dev(b))
        res = np.linalg.norm(b - p.op.M(from_dev(x, b.shape), -1)) / np.linalg.norm(b)
        assert res <= 1.05e-10, res
        assert info.reliable_updates >= 1
    finally:
        p.close()


def test_multigrid_errors():
    import torch
    from paper_2212_06635_gb300 import tm
    dims = (4, 4, 4, 4)
    u, op = _op(dims, 1971)
    ctx = _ctx(tm, u, dims)
    try:
        with pytest.raises(tm.TMError) as e:
            tm.tm_mg_create(ctx, tm.mg_params((3, 2, 2, 2), 4))
        assert e.value.status == tm.TM_ERR_ARG
        with pytest.raises(tm.TMError):
            tm.tm_mg_create(ctx, tm.mg_params((2, 2, 2, 2), 17))
        mg = tm.tm_mg_create(ctx, tm.mg_params((2, 2, 2, 2), 4, prec=tm.TM_F64))
        try:
            x = torch.zeros(256 * 24, dtype=torch.float64, device="cuda")
            b = to_dev(_full(dims, 91))
            with pytest.raises(tm.TMError) as e:       # no setup yet
                tm.tm_solve_gcr(ctx, 1, mg, tm.solve_params(), x, b)
            assert e.value.status == tm.TM_ERR_ARG
            tm.tm_mg_setup(mg, to_dev(np.stack([_full(dims, 92 + j) for j in range(4)])))
            with pytest.raises(tm.TMError) as e:       # wrong sign for this hierarchy
                tm.tm_solve_gcr(ctx, -1, mg, tm.solve_params(), x, b)
            assert e.value.status == tm.TM_ERR_ARG
            tm.tm_gauge_load(ctx, np.ascontiguousarray(u), 2.0)
            tm.tm_clover_compute(ctx, KAPPA, CSW, mu=MU)
            with pytest.raises(tm.TMError) as e:       # gauge field reloaded since the setup
                tm.tm_mg_coarse_apply(mg, x, x)
            assert e.value.status == tm.TM_ERR_STALE
            with pytest.raises(tm.TMError) as e:
                tm.tm_apply_full(ctx, 1, tm.TM_F64, np.zeros(8), x)
            assert e.value.status == tm.TM_ERR_ARG
        finally:
            tm.tm_mg_destroy(mg)
    finally:
        tm.tm_destroy(ctx)
