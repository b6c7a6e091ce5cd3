"""Run the two passes of one Schur operator a few times on a seeded lattice, for
profiling one kernel in isolation (e.g. under ncu with -k/-s/-c).

  python -m paper_2212_06635_gb300.kernel_probe --dims 32 32 32 32 --prec f16 --reps 3

Launch order: even pass x (1 + reps), then odd pass x reps (tm_kernel_times).
Prints the CUDA-event time per launch of each pass and its algorithmic GB/s.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PRECS = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
ESZ = {0: 8, 1: 4, 2: 2, 3: 2}


def ptc_grad_probe(dims, reps):
    """Time tm_ptc_grad (forward, loss, 4 weight-gradient and 3 input-gradient
    layers plus the host copies of the gradient) on a seeded pair."""
    import time
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    u = F.gauge_field(dims, 1001)
    r = F.odd_spinor(dims, 2001)
    e = F.odd_spinor(dims, 2002)
    ctx = tm.tm_create(dims, 0)
    net = tm.tm_ptc_create([1, 8, 8, 8, 1])
    try:
        tm.tm_gauge_load(ctx, u, 1.0)
        tm.tm_clover_compute(ctx, 0.14, 1.69, mu=0.0015)
        tm.tm_ptc_init(net, 0.5, 0.02, 1)
        tm.tm_ptc_grad(net, ctx, r, e)
        t0 = time.perf_counter()
        for _ in range(reps):
            tm.tm_ptc_grad(net, ctx, r, e)
        ms = (time.perf_counter() - t0) * 1e3 / max(reps, 1)
        print(f"dims {dims} PTC 1-8-8-8-1 loss + gradient: {ms:.3f} ms per pair (host inputs)")
    finally:
        tm.tm_ptc_destroy(net)
        tm.tm_destroy(ctx)


def ptc_fcg_probe(dims, iters):
    """Flexible CG preconditioned by an untrained 1-8-8-8-1 network (identity
    start), `iters` iterations on a seeded lattice: the launch sequence of the
    PTC-FCG solve, without the training."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    u = F.gauge_field(dims, 1004)
    b = F.odd_spinor(dims, 2004)
    ctx = tm.tm_create(dims, 0)
    net = tm.tm_ptc_create([1, 8, 8, 8, 1])
    try:
        tm.tm_gauge_load(ctx, u, 1.0)
        tm.tm_clover_compute(ctx, 0.1394265, 1.69, mu=0.00072)
        tm.tm_ptc_init(net, 0.5, 0.02, 1)
        bd = torch.from_numpy(b.view(np.float64).copy()).cuda()
        x = torch.zeros_like(bd)
        info = tm.tm_solve_fcg(ctx, tm.TM_MDAGM, net, tm.solve_params(tol=1e-14, maxiter=iters), x, bd, check=False)
        print(f"dims {dims} PTC-FCG {info.iters} iterations in {info.seconds:.3f} s "
              f"({1e3 * info.seconds / max(info.iters, 1):.2f} ms per iteration), "
              f"{info.reliable_updates} reliable updates, status {info.status}")
    finally:
        tm.tm_ptc_destroy(net)
        tm.tm_destroy(ctx)


def ptc_probe(dims, reps):
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    u = F.gauge_field(dims, 1001)
    b = F.odd_spinor(dims, 2001)
    ctx = tm.tm_create(dims, 0)
    net = tm.tm_ptc_create([1, 8, 8, 8, 1])
    try:
        tm.tm_gauge_load(ctx, u, 1.0)
        tm.tm_clover_compute(ctx, 0.14, 1.69, mu=0.0015)
        tm.tm_ptc_init(net, 0.5, 0.02, 1)
        bd = torch.from_numpy(b.view(np.float64).copy()).cuda()
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
        print(f"dims {dims} PTC 1-8-8-8-1 forward: {ms:.3f} ms per application")
    finally:
        tm.tm_ptc_destroy(net)
        tm.tm_destroy(ctx)


def force_bytes(dims, prec, nf, n):
    """Algorithmic bytes of one tm_force_outer launch: every field read once
    (2 n fields on V sites), the FP32 links once (12 reals per link), the FP64
    force read and written once."""
    V = int(np.prod(dims))
    site = nf * 24 * ESZ[prec] + (4 if prec >= 2 else 0)
    return 2 * n * V * site + V * 4 * 12 * 4 + 2 * V * 4 * 18 * 8


def force_probe(dims, prec, nf, n, reps, quiet=False):
    """Time tm_force_outer on n distinct (X_k, Y_k) pairs of native fields of both
    parities (seeded values, imported once and copied on the device), 1 + reps
    launches, CUDA events around the last reps.  Returns (ms per launch, bytes)."""
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    u = F.gauge_field(dims, 1002)
    ctx = tm.tm_create(dims, 0)
    try:
        tm.tm_gauge_load(ctx, u, 1.0)
        tm.tm_clover_compute(ctx, 0.14, 1.69, mu=0.0015)
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
            print(f"dims {dims} force outer products: {n} pairs, nf {nf}, fields {[k for k, v in PRECS.items() if v == prec][0]}: "
                  f"{ms * 1e3:.1f} us per launch, {b / ms / 1e6:.0f} GB/s algorithmic ({b / 1e9:.3f} GB)")
        return ms, b
    finally:
        tm.tm_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[32, 32, 32, 32])
    ap.add_argument("--prec", default="f16", choices=list(PRECS))
    ap.add_argument("--heavy", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--variant", default="direct", choices=["direct", "staged", "auto"],
                    help="stencil kernel variant of both passes (auto = tm_autotune)")
    ap.add_argument("--ptc", action="store_true",
                    help="instead: apply a 1-8-8-8-1 PTC network (1 + reps) times; each application "
                         "launches its 4 layer kernels in order")
    ap.add_argument("--ptc-fcg", type=int, default=0, metavar="ITERS",
                    help="instead: ITERS iterations of flexible CG with an untrained 1-8-8-8-1 network")
    ap.add_argument("--ptc-grad", action="store_true",
                    help="instead: loss and gradient of a 1-8-8-8-1 PTC network on one pair, (1 + reps) times")
    ap.add_argument("--force", type=int, default=0, metavar="NPAIRS",
                    help="instead: the force outer products of NPAIRS field pairs (--heavy: two flavours, "
                         "--prec: field storage f32 / f16 / bf16), (1 + reps) launches")
    a = ap.parse_args()
    import torch
    from paper_2212_06635_gb300 import tm
    from synth import fields as F
    dims = tuple(a.dims)
    if a.ptc:
        return ptc_probe(dims, a.reps)
    if a.ptc_grad:
        return ptc_grad_probe(dims, a.reps)
    if a.ptc_fcg:
        return ptc_fcg_probe(dims, a.ptc_fcg)
    if a.force:
        return force_probe(dims, PRECS[a.prec], 2 if a.heavy else 1, a.force, a.reps)
    prec = PRECS[a.prec]
    nf = 2 if a.heavy else 1
    u = F.gauge_field(dims, 1001)
    b = F.odd_spinor(dims, 2001, nf)
    ctx = tm.tm_create(dims, 0)
    try:
        tm.tm_gauge_load(ctx, u, 1.0)
        tm.tm_clover_compute(ctx, 0.14, 1.69, mu=0.0015, mubar=0.1246 if a.heavy else 0.0,
                             epsbar=0.135 if a.heavy else 0.0)
        bd = torch.from_numpy(b.view(np.float64).copy()).cuda()
        f = torch.empty(tm.tm_field_bytes(ctx, prec, nf), dtype=torch.uint8, device="cuda")
        tm.tm_field_import(ctx, prec, nf, f, bd)
        op = tm.TM_QH if a.heavy else tm.TM_QHAT_PLUS
        if a.variant == "auto":
            tm.tm_autotune(ctx, prec, nf)
        elif prec != 0:
            v = 1 if a.variant == "staged" else 0
            tm.tm_set_tuning(ctx, prec, nf, v, v)
        t1, t2 = tm.tm_kernel_times(ctx, op, prec, f, a.reps)
        vh = int(np.prod(dims)) // 2
        esz = ESZ[prec]
        sc = 4 if prec >= 2 else 0
        links = 8 * (12 if prec in (1, 3) else 18)
        r1, r2 = (links + 240, links + 216) if a.heavy else (links + 192, links + 144)
        s1, s2 = (2, 3)
        b1 = (r1 * esz + s1 * sc) * vh
        b2 = (r2 * esz + s2 * sc) * vh
        print(f"dims {dims} prec {a.prec} nf {nf}: even pass {t1 * 1e3:.1f} us {b1 / t1 / 1e6:.0f} GB/s; "
              f"odd pass {t2 * 1e3:.1f} us {b2 / t2 / 1e6:.0f} GB/s")
    finally:
        tm.tm_destroy(ctx)


if __name__ == "__main__":
    main()
