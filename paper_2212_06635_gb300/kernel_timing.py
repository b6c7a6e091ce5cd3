"""CUDA-event timings of single library entry points on seeded inputs, with the
algorithmic bytes each launch moves.  bench.py takes its per-kernel figures from
here, and the ncu captures under profiles/ run these same launch sequences.

  python -m paper_2212_06635_gb300.kernel_timing --dims 32 32 32 32 --prec f16 --reps 3
      even pass x (1 + reps), then odd pass x reps (tm_kernel_times)
  ... --heavy                     the two-flavour passes
  ... --force NPAIRS [--heavy]    tm_force_outer on NPAIRS field pairs, 1 + reps launches
  ... --ptc                       a 1-8-8-8-1 PTC network applied 1 + reps times
  ... --ptc-grad                  loss and gradient of that network, 1 + reps times
  ... --ptc-fcg ITERS             ITERS iterations of PTC-preconditioned flexible CG
  ... --solve [--solves N] [--delta D]
                                  N mixed-precision CG solves (--prec storage) to 1e-10
  ... --dw [--heavy]              the normal operator on FP64 fields, native FP64 and
                                  double-word (the reliable updates' operator), 1 + reps each
  ... --multishift                a 12-shift heavy-doublet multishift solve (--prec storage)
  ... --mg ITERS                  multigrid setup and ITERS multigrid-preconditioned GCR iterations
  ... --fma                       measured FP64 and FP32 FMA rates of the CUDA cores
  ... --batch batched|sequential  the uneven batch of 24 light solves (mixed FP16 CG)
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PRECS = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
ESZ = {0: 8, 1: 4, 2: 2, 3: 2}
KAPPA, CSW, MU, MUBAR, EPSBAR = 0.14, 1.69, 0.0015, 0.1246, 0.135


def pass_bytes(prec, nf, vh):
    """Algorithmic bytes of the even and the odd pass of one Schur operator
    (each field read or written once): links 8 x 12 reals (FP32, FP16) or 18
    (FP64, BF16); light even pass psi 24 + inverse blocks 144 + out 24 reals, odd
    pass t_e 24 + psi 24 + clover 72 + out 24; heavy spinors 48 reals, and the
    even inverse counted as its 144-real minimum (the hermitian A and D_h of both
    chiralities); 16-bit spinors add one FP32 scale per site and spinor access."""
    esz = ESZ[prec]
    sc = 4 if prec >= 2 else 0
    links = 8 * (12 if prec in (1, 3) else 18)
    r1, r2 = (links + 240, links + 216) if nf == 2 else (links + 192, links + 144)
    return (r1 * esz + 2 * sc) * vh, (r2 * esz + 3 * sc) * vh


def _ctx(tm, dims, heavy, seed=1001):
    from synth import fields as F
    ctx = tm.tm_create(dims, 0)
    tm.tm_gauge_load(ctx, F.gauge_field(dims, seed), 1.0)
    tm.tm_clover_compute(ctx, KAPPA, CSW, mu=MU, mubar=MUBAR if heavy else 0.0, epsbar=EPSBAR if heavy else 0.0)
    return ctx


def stencil_passes(dims, prec, nf, reps, variant="direct", quiet=False):
    """CUDA-event time per launch of the two passes of Q_hat (light) or Q_hat_h
    (heavy).  Returns (even ms, odd ms, even bytes, odd bytes)."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    ctx = _ctx(tm, dims, nf == 2)
    try:
        bd = torch.from_numpy(F.odd_spinor(dims, 2001, nf).view(np.float64).copy()).cuda()
        f = torch.empty(tm.tm_field_bytes(ctx, prec, nf), dtype=torch.uint8, device="cuda")
        tm.tm_field_import(ctx, prec, nf, f, bd)
        op = tm.TM_QH if nf == 2 else tm.TM_QHAT_PLUS
        if variant == "auto":
            tm.tm_autotune(ctx, prec, nf)
        elif prec != 0:
            v = 1 if variant == "staged" else 0
            tm.tm_set_tuning(ctx, prec, nf, v, v)
        t1, t2 = tm.tm_kernel_times(ctx, op, prec, f, reps)
        b1, b2 = pass_bytes(prec, nf, int(np.prod(dims)) // 2)
        if not quiet:
            name = [k for k, v in PRECS.items() if v == prec][0]
            print(f"dims {dims} prec {name} nf {nf}: even pass {t1 * 1e3:.1f} us {b1 / t1 / 1e6:.0f} GB/s; "
                  f"odd pass {t2 * 1e3:.1f} us {b2 / t2 / 1e6:.0f} GB/s")
        return t1, t2, b1, b2
    finally:
        tm.tm_destroy(ctx)


def double_word(dims, nf, reps, quiet=False):
    """CUDA-event time of the normal operator (M_hat^dag M_hat light, Q_hat_h
    Q_hat_h^dag heavy) on native FP64 fields: native FP64 arithmetic
    (tm_apply_Mhat, TM_F64) against double-word arithmetic (tm_apply_Mhat_dw,
    conversions in and out included).  Returns (FP64 ms, double-word ms)."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    ctx = _ctx(tm, dims, nf == 2)
    try:
        src = torch.from_numpy(F.odd_spinor(dims, 2002, nf).view(np.float64).copy()).cuda()
        a = torch.empty(tm.tm_field_bytes(ctx, 0, nf), dtype=torch.uint8, device="cuda")
        o = torch.empty_like(a)
        tm.tm_field_import(ctx, 0, nf, a, src)
        op = tm.TM_QH_SQ if nf == 2 else tm.TM_MDAGM
        res = []
        for f in (lambda: tm.tm_apply_Mhat(ctx, op, 0, o, a), lambda: tm.tm_apply_Mhat_dw(ctx, op, o, a)):
            f()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                f()
            e1.record()
            torch.cuda.synchronize()
            res.append(e0.elapsed_time(e1) / max(reps, 1))
        if not quiet:
            print(f"dims {dims} nf {nf} normal operator on FP64 fields: native FP64 {res[0] * 1e3:.1f} us, "
                  f"double-word {res[1] * 1e3:.1f} us ({res[0] / res[1]:.2f}x)")
        return tuple(res)
    finally:
        tm.tm_destroy(ctx)


def force_bytes(dims, prec, nf, n):
    """Algorithmic bytes of one tm_force_outer launch: every field read once
    (2 n fields on V sites), the FP32 links once (12 reals per link), the FP64
    force read and written once."""
    V = int(np.prod(dims))
    site = nf * 24 * ESZ[prec] + (4 if prec >= 2 else 0)
    return 2 * n * V * site + V * 4 * 12 * 4 + 2 * V * 4 * 18 * 8


def force_outer(dims, prec, nf, n, reps, quiet=False):
    """tm_force_outer on n distinct (X_k, Y_k) pairs of native fields of both
    parities (seeded values, imported once and copied on the device), 1 + reps
    launches, CUDA events around the last reps.  Returns (ms per launch, bytes)."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    ctx = _ctx(tm, dims, False, seed=1002)
    try:
        nbytes = tm.tm_field_bytes(ctx, prec, nf)
        seeds = []
        for s in range(4):
            src = torch.from_numpy(F.odd_spinor(dims, 2100 + s, nf).view(np.float64).copy()).cuda()
            f = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            tm.tm_field_import(ctx, prec, nf, f, src)
            seeds.append(f)
            del src
        fields = [[seeds[(2 * w + p) % 4].clone() for p in range(2)] for w in range(2 * n)]
        xs, ys = fields[:n], fields[n:]
        c = [1.0 / (1 + k) for k in range(n)]
        force = torch.zeros(int(np.prod(dims)) * 4 * 18, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        tm.tm_force_outer(ctx, prec, nf, c, xs, ys, force)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            tm.tm_force_outer(ctx, prec, nf, c, xs, ys, force)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(reps, 1)
        b = force_bytes(dims, prec, nf, n)
        if not quiet:
            name = [k for k, v in PRECS.items() if v == prec][0]
            print(f"dims {dims} force outer products: {n} pairs, nf {nf}, fields {name}: "
                  f"{ms * 1e3:.1f} us per launch, {b / ms / 1e6:.0f} GB/s algorithmic ({b / 1e9:.3f} GB)")
        return ms, b
    finally:
        tm.tm_destroy(ctx)


def ptc_forward(dims, reps, quiet=False):
    """A 1-8-8-8-1 network (identity start) applied 1 + reps times to an FP32
    field; CUDA events around the last reps.  Returns ms per application."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    ctx = _ctx(tm, dims, False)
    net = tm.tm_ptc_create([1, 8, 8, 8, 1])
    try:
        tm.tm_ptc_init(net, 0.5, 0.02, 1)
        bd = torch.from_numpy(F.odd_spinor(dims, 2001).view(np.float64).copy()).cuda()
        f = torch.empty(tm.tm_field_bytes(ctx, tm.TM_F32, 1), dtype=torch.uint8, device="cuda")
        o = torch.empty_like(f)
        tm.tm_field_import(ctx, tm.TM_F32, 1, f, bd)
        tm.tm_ptc_apply(net, ctx, o, f)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            tm.tm_ptc_apply(net, ctx, o, f)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(reps, 1)
        if not quiet:
            print(f"dims {dims} PTC 1-8-8-8-1 forward: {ms:.3f} ms per application")
        return ms
    finally:
        tm.tm_ptc_destroy(net)
        tm.tm_destroy(ctx)


def ptc_grad(dims, reps, quiet=False):
    """tm_ptc_grad (forward, loss, weight- and input-gradient layers and the host
    copies of the gradient) on one seeded pair, 1 + reps times.  Returns ms per pair."""
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    r = F.odd_spinor(dims, 2001)
    e = F.odd_spinor(dims, 2002)
    ctx = _ctx(tm, dims, False)
    net = tm.tm_ptc_create([1, 8, 8, 8, 1])
    try:
        tm.tm_ptc_init(net, 0.5, 0.02, 1)
        tm.tm_ptc_grad(net, ctx, r, e)
        t0 = time.perf_counter()
        for _ in range(reps):
            tm.tm_ptc_grad(net, ctx, r, e)
        ms = (time.perf_counter() - t0) * 1e3 / max(reps, 1)
        if not quiet:
            print(f"dims {dims} PTC 1-8-8-8-1 loss + gradient: {ms:.3f} ms per pair (host inputs)")
        return ms
    finally:
        tm.tm_ptc_destroy(net)
        tm.tm_destroy(ctx)


def ptc_fcg(dims, iters, quiet=False):
    """Flexible CG preconditioned by an untrained 1-8-8-8-1 network (identity
    start), `iters` iterations: the launch sequence of a PTC-FCG solve."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    b = F.odd_spinor(dims, 2004)
    ctx = tm.tm_create(dims, 0)
    net = tm.tm_ptc_create([1, 8, 8, 8, 1])
    try:
        tm.tm_gauge_load(ctx, F.gauge_field(dims, 1004), 1.0)
        tm.tm_clover_compute(ctx, 0.1394265, CSW, mu=0.00072)
        tm.tm_ptc_init(net, 0.5, 0.02, 1)
        bd = torch.from_numpy(b.view(np.float64).copy()).cuda()
        x = torch.zeros_like(bd)
        info = tm.tm_solve_fcg(ctx, tm.TM_MDAGM, net, tm.solve_params(tol=1e-14, maxiter=iters), x, bd, check=False)
        if not quiet:
            print(f"dims {dims} PTC-FCG {info.iters} iterations in {info.seconds:.3f} s "
                  f"({1e3 * info.seconds / max(info.iters, 1):.2f} ms per iteration), "
                  f"{info.reliable_updates} reliable updates, status {info.status}")
        return info
    finally:
        tm.tm_ptc_destroy(net)
        tm.tm_destroy(ctx)


def cg_solve(dims, prec, quiet=False, delta=0.0, solves=1):
    """CG solves of M_hat^dag M_hat to true rel. res. 1e-10 with the given sloppy
    storage (FP64: plain FP64 CG) and reliable-update threshold (0: the library's
    default), from a zero guess: the launch sequence of the solver's stencil and
    BLAS-1 kernels.  Returns the last solve's info."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    ctx = _ctx(tm, dims, False)
    try:
        if prec != 0:
            tm.tm_autotune(ctx, prec, 1)
        bd = torch.from_numpy(F.odd_spinor(dims, 2001).view(np.float64).copy()).cuda()
        for _ in range(solves):
            x = torch.zeros_like(bd)
            info = tm.tm_solve_cg(ctx, tm.TM_MDAGM, tm.solve_params(tol=1e-10, sloppy=prec, delta=delta), x, bd,
                                  check=False)
            if not quiet:
                print(f"dims {dims} CG sloppy {prec} delta {delta}: {info.iters} iterations, "
                      f"{info.reliable_updates} reliable updates, {info.seconds:.4f} s, "
                      f"residual {info.true_rel_res:.2e}")
        return info
    finally:
        tm.tm_destroy(ctx)


def multishift(dims, prec, nshift=12, quiet=False):
    """One heavy-doublet multishift solve (Q_h Q_h^dag, nshift shifts log-spaced in
    [1e-5, 1] x 1.02 lambda_max) in storage prec, refined shift by shift to 1e-10:
    the launch sequence of the multishift update kernels."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    ctx = _ctx(tm, dims, True, seed=1002)
    try:
        if prec != 0:
            tm.tm_autotune(ctx, prec, 2)
        lam = 1.02 * tm.tm_power_iteration(ctx, tm.TM_QH_SQ, 50)
        shifts = [lam * 10.0 ** (-5 + 5 * k / (nshift - 1)) for k in range(nshift)]
        bd = torch.from_numpy(F.odd_spinor(dims, 2002, 2).view(np.float64).copy()).cuda()
        xs = [torch.zeros_like(bd) for _ in shifts]
        infos = tm.tm_solve_multishift(ctx, tm.TM_QH_SQ, shifts, xs, bd, tm.solve_params(tol=1e-10, sloppy=prec),
                                       check=False)
        if not quiet:
            print(f"dims {dims} multishift {nshift} shifts, storage {prec}: {infos[0].seconds:.4f} s, "
                  f"iterations {[i.iters for i in infos]}")
        return infos
    finally:
        tm.tm_destroy(ctx)


def mg_solve(dims, block=(4, 4, 4, 4), nvec=12, setup=100, smooth=8, maxiter=20, quiet=False):
    """Multigrid setup (FP32) and a bounded multigrid-preconditioned GCR solve of
    the full operator: the launch sequence of the multigrid kernels."""
    import torch
    from paper_2212_06635_gb300 import tm
    ctx = _ctx(tm, dims, False, seed=1004)
    mg = None
    try:
        V = int(np.prod(dims))
        g = torch.Generator(device="cuda")
        g.manual_seed(7)
        init = torch.randn(nvec * V * 24, dtype=torch.float64, device="cuda", generator=g)
        b = torch.randn(V * 24, dtype=torch.float64, device="cuda", generator=g)
        mg = tm.tm_mg_create(ctx, tm.mg_params(block, nvec, setup, smooth, 1, tm.TM_F32, 0.1, 30, 16))
        t0 = time.perf_counter()
        tm.tm_mg_setup(mg, init)
        ts = time.perf_counter() - t0
        del init
        x = torch.zeros_like(b)
        info = tm.tm_solve_gcr(ctx, 1, mg, tm.solve_params(tol=1e-10, maxiter=maxiter, sloppy=tm.TM_F32, chunk=16),
                               x, b, check=False)
        if not quiet:
            print(f"dims {dims} multigrid setup {ts:.3f} s; GCR {info.iters} iterations {info.seconds:.3f} s "
                  f"residual {info.true_rel_res:.2e}")
        return info
    finally:
        if mg is not None:
            tm.tm_mg_destroy(mg)
        tm.tm_destroy(ctx)


def batch_solve(sequential=False, chunk=16, quiet=False):
    """The uneven batch of 24 light problems (6 each of 8^3x16, 12^3x24, 16^3x32,
    24^3x48), mixed FP16 CG to 1e-10: one batched solve (or the 24 solves one
    after another): the launch sequence of the batched kernels."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import configs as CFG
    from synth import fields as F
    ws = CFG.batch_workloads()
    ctxs, bs, xs = [], [], []
    try:
        for w in ws:
            c = tm.tm_create(w.dims, 0)
            ctxs.append(c)
            tm.tm_gauge_load(c, F.gauge_field(w.dims, w.link_seed, workers=1), 1.0)
            tm.tm_clover_compute(c, w.kappa, w.csw, mu=w.mu, bc_t=w.bc_t)
            tm.tm_autotune(c, tm.TM_F16, 1)
            bs.append(torch.from_numpy(F.odd_spinor(w.dims, w.rhs_seed).view(np.float64).copy()).cuda())
            xs.append(torch.zeros_like(bs[-1]))
        sp = tm.solve_params(tol=1e-10, sloppy=tm.TM_F16, chunk=chunk)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if sequential:
            infos = [tm.tm_solve_cg(c, tm.TM_MDAGM, sp, x, b, check=False) for c, x, b in zip(ctxs, xs, bs)]
        else:
            infos = tm.tm_solve_batch(ctxs, tm.TM_MDAGM, sp, xs, bs, check=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if not quiet:
            print(f"uneven batch of {len(ws)}, {'sequential' if sequential else 'batched'}, chunk {chunk}: {dt:.4f} s, "
                  f"iterations {[i.iters for i in infos]}, reliable updates {[i.reliable_updates for i in infos]}")
        return dt
    finally:
        for c in ctxs:
            tm.tm_destroy(c)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[32, 32, 32, 32])
    ap.add_argument("--prec", default="f16", choices=list(PRECS))
    ap.add_argument("--heavy", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--variant", default="direct", choices=["direct", "staged", "auto"],
                    help="stencil kernel variant of both passes (auto = tm_autotune)")
    ap.add_argument("--ptc", action="store_true")
    ap.add_argument("--ptc-fcg", type=int, default=0, metavar="ITERS")
    ap.add_argument("--ptc-grad", action="store_true")
    ap.add_argument("--force", type=int, default=0, metavar="NPAIRS")
    ap.add_argument("--solve", action="store_true")
    ap.add_argument("--multishift", action="store_true")
    ap.add_argument("--delta", type=float, default=0.0, help="--solve: reliable-update threshold (0: default)")
    ap.add_argument("--solves", type=int, default=1, help="--solve: solves in a row (the first one warms up)")
    ap.add_argument("--mg", type=int, default=0, metavar="ITERS",
                    help="multigrid setup, then ITERS iterations of multigrid-preconditioned GCR")
    ap.add_argument("--setup", type=int, default=100, help="--mg: minimal-residual steps per near-null vector")
    ap.add_argument("--batch", choices=["batched", "sequential"], default=None,
                    help="the uneven batch of 24 light solves, batched or one after another")
    ap.add_argument("--chunk", type=int, default=16, help="--batch: iterations between host checks")
    ap.add_argument("--fma", action="store_true", help="measured FP64 and FP32 FMA rates")
    ap.add_argument("--dw", action="store_true",
                    help="normal operator on FP64 fields: native FP64 against double-word arithmetic")
    a = ap.parse_args()
    dims = tuple(a.dims)
    prec = PRECS[a.prec]
    nf = 2 if a.heavy else 1
    if a.ptc:
        ptc_forward(dims, a.reps)
    elif a.ptc_grad:
        ptc_grad(dims, a.reps)
    elif a.ptc_fcg:
        ptc_fcg(dims, a.ptc_fcg)
    elif a.force:
        force_outer(dims, prec, nf, a.force, a.reps)
    elif a.solve:
        cg_solve(dims, prec, delta=a.delta, solves=a.solves)
    elif a.multishift:
        multishift(dims, prec)
    elif a.mg:
        mg_solve(dims, setup=a.setup, maxiter=a.mg)
    elif a.batch:
        batch_solve(sequential=a.batch == "sequential", chunk=a.chunk)
    elif a.dw:
        double_word(dims, nf, a.reps)
    elif a.fma:
        from paper_2212_06635_gb300 import tm
        for p, name in ((0, "FP64"), (1, "FP32")):
            print(f"{name} FMA rate: {tm.tm_fma_rate(0, p) / 1e12:.3f} TFLOP/s")
    else:
        stencil_passes(dims, prec, nf, a.reps, a.variant)


if __name__ == "__main__":
    main()
