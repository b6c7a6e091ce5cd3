#!/usr/bin/env python
"""Benchmark of the even-odd twisted-mass clover solver path on GB300.

Workload: light doublet on a 32^3x64 lattice (kappa 0.1400, csw 1.69, mu 0.0015,
antiperiodic time), seeded synthetic SU(3) links (mean plaquette 0.59) and a
complex-Gaussian right-hand side.

One step = one application of the normal operator M_hat^dag M_hat = Q_hat_- Q_hat_+
(two Schur operator applications, four kernels) in the mixed solver's storage
format (FP16 fields with one FP32 scale per site, FP32 arithmetic).  The value is
M_hat HBM GB/s: algorithmic bytes of the M_hat applications / device time.  The
same JSON line carries the second half of the metric: seconds to true relative
residual 1e-10 of the chosen form (mixed-precision CG) and of plain FP64 CG on
the same GPU.

Before that headline line, one JSON line holds the records of the other
workloads: the reliable updates' operator (native FP64 against double-word
arithmetic) at 32^3x64, the heavy-doublet multishift at 24^3x48, the uneven batch, the force
outer products, the rational correction term, the two-level multigrid of the
full operator at 48^3x96 against the even-odd mixed CG route, and the PTC
network trained on 2048 solver-generated pairs from 8 configurations at
48^3x96 inside flexible CG.  The headline line repeats their times to solution
under `workload_summary`.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]
                  [--no-extra] [--no-mg] [--no-ptc] [--ptc-quick] [--variant direct|staged]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import configs as CFG  # noqa: E402
from synth import fields as F  # noqa: E402

METRIC = "Mhat HBM GB/s (% peak); seconds to rel res 1e-10, chosen form vs plain FP64 CG"
W = CFG.LIGHT_32
CPU_SAMPLE_DIMS = (16, 16, 16, 16)
ESZ = {0: 8, 1: 4, 2: 2, 3: 2}


def mhat_bytes_per_site(prec):
    """Algorithmic bytes of one M_hat application per odd site (each field read or
    written once per pass): even pass 8 links + psi 24 + inverse blocks 144 +
    t_e 24 reals, odd pass 8 links + t_e 24 + psi 24 + clover 72 + out 24 reals.
    A link is 12 reals (two rows) in FP32 and FP16 storage and 18 in FP64 and BF16; 16-bit
    spinors add one FP32 scale per site per spinor access."""
    esz = ESZ[prec]
    scale = 4 if prec in (2, 3) else 0
    links = 8 * (12 if prec in (1, 3) else 18)
    k1 = (links + 192) * esz + 2 * scale
    k2 = (links + 144) * esz + 3 * scale
    return k1, k2


def max_over_ranks(seconds_or_ms, device=None):
    """Largest value over the ranks of the default process group (identity when
    no group is initialised).  device: where the reduction tensor lives (a CUDA
    device for NCCL, None = CPU for gloo)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return float(seconds_or_ms)
    t = torch.tensor([float(seconds_or_ms)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbs(world, step_bytes, steps, seconds):
    """Whole-job GB/s: every rank runs its own replica (weak scaling); the job
    processed world * steps steps in the slowest rank's time."""
    return world * step_bytes * steps / seconds / 1e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


KERNEL_SOURCES = ["tm_internal.h", "fastdiv.h", "tm_kernels.h", "dslash_common.cuh", "dslash.cu", "dslash_staged.cu"]


def kernel_sources_sha256():
    """Hash of every source the stencil kernels are compiled from."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2212_06635_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_from_profile(kernel_tag):
    """DRAM bytes per launch recorded by ncu for the current kernel source, else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        entry = rec.get(kernel_tag)
        if entry and entry.get("kernel_sources_sha256") == kernel_sources_sha256():
            return float(entry["dram_bytes_per_launch_full_size"])
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
MHAT_FLOP_PER_SITE = 3792     # 2 Wilson hops (1320 each) + 2 6x6-pair matvecs (552 each) + axpy 48


def cpu_oracle_steps(nsteps, dims=CPU_SAMPLE_DIMS):
    """Time the FP64 oracle applying M_hat^dag M_hat on a sub-lattice of the same
    workload in this process (one core); returns (GB/s in FP64 algorithmic
    bytes, seconds per step)."""
    from oracle import dirac as D
    u = F.gauge_field(dims, W.link_seed, workers=1)
    op = D.TwistedMassClover(u, dims, W.kappa, W.csw, mu=W.mu, bc_t=W.bc_t)
    op.inv_even_light(+1)
    op.inv_even_light(-1)
    b = F.odd_spinor(dims, W.rhs_seed)
    vh = op.geo.V // 2
    k1, k2 = mhat_bytes_per_site(0)
    times = []
    for _ in range(nsteps):
        t0 = time.perf_counter()
        op.MdagM(b)
        times.append(time.perf_counter() - t0)
    sec = float(np.mean(times))
    return 2 * (k1 + k2) * vh / sec / 1e9, sec


_CPU_BARRIER = None


def _cpu_init(barrier):
    global _CPU_BARRIER
    _CPU_BARRIER = barrier


def _cpu_replica(job):
    """One host process: the oracle's M_hat^dag M_hat on its own right-hand side
    (warmup untimed steps, then steps timed after every process is ready)."""
    dims, rhs_seed, warmup, steps = job
    from oracle import dirac as D
    u = F.gauge_field(dims, W.link_seed, workers=1)
    op = D.TwistedMassClover(u, dims, W.kappa, W.csw, mu=W.mu, bc_t=W.bc_t)
    op.inv_even_light(+1)
    op.inv_even_light(-1)
    b = F.odd_spinor(dims, rhs_seed)
    for _ in range(warmup):
        op.MdagM(b)
    _CPU_BARRIER.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        op.MdagM(b)
    return time.perf_counter() - t0


def cpu_oracle_parallel(warmup, steps, nproc=None, dims=CPU_SAMPLE_DIMS):
    """The oracle on every host core: nproc spawned processes (one numpy thread
    each) apply M_hat^dag M_hat to independent right-hand sides of the same
    sub-lattice at the same time, the oracle's arithmetic unchanged.  Returns
    (aggregate GB/s, processes, seconds of the slowest process per step)."""
    import multiprocessing as mp
    nproc = nproc or min(os.cpu_count() or 1, 32)
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(nproc)
        jobs = [(dims, W.rhs_seed + 100 * k, warmup, steps) for k in range(nproc)]
        with ctx.Pool(nproc, initializer=_cpu_init, initargs=(barrier,)) as pool:
            secs = pool.map(_cpu_replica, jobs, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    vh = int(np.prod(dims)) // 2
    k1, k2 = mhat_bytes_per_site(0)
    tmax = max(secs)
    return nproc * steps * 2 * (k1 + k2) * vh / tmax / 1e9, nproc, tmax / steps


def cpu_solve_4x4():
    """Seconds of the oracle's FP64 CG on the 4^4 workload (M_hat^dag M_hat to
    1e-12), one core, and its iteration count."""
    from oracle import dirac as D
    from oracle import solvers as S
    w = CFG.LIGHT_4
    op = D.TwistedMassClover(F.gauge_field(w.dims, w.link_seed, workers=1), w.dims, w.kappa, w.csw, mu=w.mu,
                             bc_t=w.bc_t)
    b = F.odd_spinor(w.dims, w.rhs_seed)
    t0 = time.perf_counter()
    op.inv_even_light(+1)
    op.inv_even_light(-1)
    x, it = S.cg(op.MdagM, b, tol=w.tol)
    return time.perf_counter() - t0, it


def cpu_baseline_record(args, fp64_iters=None):
    """The cpu_baseline object: the oracle on all host cores (replicas of the
    sub-lattice), one core alone, the 4^4 CPU solve, and the 32^3x64 FP64 CG
    extrapolated from the one-core step time (labelled as such)."""
    gbs, nproc, sec = cpu_oracle_parallel(1, 2)
    gbs1, sec1 = cpu_oracle_steps(2)
    s4, it4 = cpu_solve_4x4()
    lat = "x".join(map(str, CPU_SAMPLE_DIMS))
    rec = {"value": round(gbs, 4), "unit": "GB/s", "cores": nproc, "kind": "oracle",
           "sample": f"FP64 numpy oracle as it stands, M_hat^dag M_hat on a {lat} sub-lattice of the same action: "
                     f"{nproc} processes on independent right-hand sides, 2 timed steps each "
                     f"({sec:.2f} s per step); host cores of this box",
           "one_core": {"value": round(gbs1, 4), "unit": "GB/s", "seconds_per_step": round(sec1, 3)},
           "host": {"cpu_count": os.cpu_count(), "machine": os.uname().machine},
           "cpu_fp64_cg_4x4x4x4": {"seconds": round(s4, 3), "iters": it4, "tol": CFG.LIGHT_4.tol}}
    if fp64_iters:
        vol = W.volume / int(np.prod(CPU_SAMPLE_DIMS))
        rec["cpu_fp64_cg_32x64_extrapolated"] = {
            "seconds": round(sec1 * vol * fp64_iters, 1), "iters": fp64_iters,
            "how": "extrapolated, not run: one-core step time x volume ratio x the GPU FP64 CG iteration count"}
    return rec


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    t0 = time.perf_counter()
    gbs, nproc, sec = cpu_oracle_parallel(args.warmup, args.steps)
    wall = time.perf_counter() - t0
    sample = (f"oracle (numpy FP64, as it stands) M_hat^dag M_hat on a {'x'.join(map(str, CPU_SAMPLE_DIMS))} "
              f"sub-lattice of the same action: {nproc} host processes on independent right-hand sides, "
              f"{args.warmup} untimed + {args.steps} timed steps each")
    line = {"impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": W.name, "lattice": list(CPU_SAMPLE_DIMS),
                                            "step": "M_hat^dag M_hat (2 M_hat), FP64 oracle, one per host process"},
            "gflops": round(gbs / (2 * sum(mhat_bytes_per_site(0))) * 2 * MHAT_FLOP_PER_SITE, 4),
            "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": nproc, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2212_06635_gb300 import tm

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    prec = {"f16": tm.TM_F16, "bf16": tm.TM_BF16, "f32": tm.TM_F32}[args.storage]

    u = F.gauge_field(W.dims, W.link_seed)
    b = F.odd_spinor(W.dims, W.rhs_seed)
    vh = W.volume // 2
    ctx = tm.tm_create(W.dims, local_rank)
    try:
        tm.tm_gauge_load(ctx, u, 1.0)
        tm.tm_clover_compute(ctx, W.kappa, W.csw, mu=W.mu, bc_t=W.bc_t)
        if args.variant == "auto":
            tuning = tm.tm_autotune(ctx, prec, 1)
        else:   # a fixed stencil variant (a profiler run times kernels unlike a plain one)
            v = 1 if args.variant == "staged" else 0
            tm.tm_set_tuning(ctx, prec, 1, v, v)
            tuning = (v, v)
        bd = torch.from_numpy(b.view(np.float64).copy()).to(dev)
        nbytes = tm.tm_field_bytes(ctx, prec, 1)
        fin = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        fout = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        tm.tm_field_import(ctx, prec, 1, fin, bd)
        torch.cuda.synchronize()
        k1b, k2b = mhat_bytes_per_site(prec)
        step_bytes = 2 * (k1b + k2b) * vh
        stream = torch.cuda.current_stream()

        def barrier():
            if dist:
                tdist.barrier()

        # ---- device-resident steps -----------------------------------------
        for _ in range(args.warmup):
            tm.tm_apply_Mhat(ctx, tm.TM_MDAGM, prec, fout, fin)
        torch.cuda.synchronize()
        clk = ClockSampler(torch.cuda.current_device() if not dist else local_rank)
        clk.start()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            tm.tm_apply_Mhat(ctx, tm.TM_MDAGM, prec, fout, fin)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = clk.stop()
        ms = max_over_ranks(e0.elapsed_time(e1), dev if dist else None)
        value = aggregate_gbs(world, step_bytes, args.steps, ms * 1e-3)

        # ---- dominant kernel against the roofline ------------------------------
        t1, t2 = tm.tm_kernel_times(ctx, tm.TM_QHAT_PLUS, prec, fin, reps=50)
        kernels = {"even pass (hop + inverse blocks)": (t1, k1b * vh), "odd pass (hop + clover + g5)": (t2, k2b * vh)}
        dom = max(kernels, key=lambda k: kernels[k][0])
        dms, dbytes = kernels[dom]
        peak, peak_kind = peaks()
        achieved = dbytes / (dms * 1e-3) / 1e9
        tag = f"{'k1' if dom.startswith('even') else 'k2'}_{args.storage}"
        traffic = traffic_from_profile(tag)

        # ---- end to end through the C ABI with host buffers ---------------------
        # Every step uploads its canonical FP64 input from pinned host memory
        # (tm_field_import), applies M_hat^dag M_hat and downloads the canonical
        # result (tm_field_export).  Steps are pipelined as a serving loop would:
        # uploads on one stream, the operator on a second, downloads on a third, two
        # steps in flight, ordered by events.
        hins = [torch.empty(vh * 24, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        for h in hins:
            h.copy_(torch.from_numpy(b.view(np.float64).reshape(-1)))
        houts = [torch.empty_like(hins[0], pin_memory=True) for _ in range(2)]
        fins = [fin, torch.empty_like(fin)]
        fouts = [fout, torch.empty_like(fout)]
        s_in, s_op, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_op = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def e2e_steps(n):
            for k in range(n):
                i = k % 2
                if k >= 2:
                    s_in.wait_event(ev_op[i])        # fins[i] read by the operator two steps back
                tm.tm_field_import(ctx, prec, 1, fins[i], hins[i], stream=s_in)
                ev_in[i].record(s_in)
                s_op.wait_event(ev_in[i])
                if k >= 2:
                    s_op.wait_event(ev_out[i])       # fouts[i] read by the download two steps back
                tm.tm_apply_Mhat(ctx, tm.TM_MDAGM, prec, fouts[i], fins[i], stream=s_op)
                ev_op[i].record(s_op)
                s_out.wait_event(ev_op[i])
                tm.tm_field_export(ctx, prec, 1, houts[i], fouts[i], stream=s_out)
                ev_out[i].record(s_out)
            torch.cuda.synchronize()

        e2e_steps(max(2, args.warmup // 2))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps(args.steps)
        e2e_s = max_over_ranks(time.perf_counter() - t0, dev if dist else None)
        e2e = aggregate_gbs(world, step_bytes, args.steps, e2e_s)

        # ---- seconds to true rel res 1e-10: chosen form vs FP64 CG ----------------
        tts = {}
        if not args.no_solve:
            forms = [("chosen", prec, "mixed-precision CG: %s storage, FP32 math, double-word reliable updates, FP64 final residual"
                      % args.storage)]
            if not args.no_fp64:
                forms.append(("fp64_cg", tm.TM_F64, "plain FP64 CG"))
            for name, sl, desc in forms:
                x = torch.zeros_like(bd)
                sp = tm.solve_params(tol=W.tol, sloppy=sl, maxiter=args.maxiter)
                torch.cuda.synchronize()
                info = tm.tm_solve_cg(ctx, tm.TM_MDAGM, sp, x, bd, check=False)
                tts[name] = {"form": desc, "seconds": round(info.seconds, 4), "iters": info.iters,
                             "reliable_updates": info.reliable_updates, "true_rel_res": info.true_rel_res,
                             "status": tm.STATUS_NAMES[info.status]}
            if "fp64_cg" in tts and tts["chosen"]["seconds"] > 0:
                tts["speedup_vs_fp64_cg"] = round(tts["fp64_cg"]["seconds"] / tts["chosen"]["seconds"], 3)
        dw_rec = None
        if rank == 0 and not args.no_extra:
            dw_rec = run_reliable_update_operator(tm, ctx, bd, dev)
    finally:
        tm.tm_destroy(ctx)

    extra = {}
    if dw_rec is not None:
        extra["reliable_update_operator_32x64"] = dw_rec
    if rank == 0 and not args.no_extra:
        extra["multishift_heavy_24x48"] = run_multishift(tm, args)
        extra["batch_uneven_24"] = run_batch(tm, args)
        extra["force_outer_heavy_24x48"] = run_force(args, peak)
        extra["rational_correction_heavy_24x48"] = run_rational(tm, args)
    if rank == 0 and not args.no_mg:
        try:
            extra["mg_gcr_48x96"] = run_mg(tm, args)
        except Exception as e:  # recorded in the line, not swallowed
            extra["mg_gcr_48x96"] = {"error": repr(e)}
    if rank == 0 and not args.no_ptc:
        try:
            extra["ptc_fcg_48x96"] = run_ptc(tm, args)
        except Exception as e:  # recorded in the line, not swallowed: the M_hat figures above stand
            extra["ptc_fcg_48x96"] = {"error": repr(e)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_record(args, tts.get("fp64_cg", {}).get("iters"))
    if rank == 0:
        # the full per-workload records go on their own line before the headline,
        # so that the headline (the last line) stays short
        print(json.dumps({"workloads": extra}), flush=True)
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": W.name, "lattice": list(W.dims), "kappa": W.kappa, "csw": W.csw, "mu": W.mu,
                       "storage": args.storage, "math": "f32",
                       "step": "M_hat^dag M_hat = Q_hat_- Q_hat_+ (2 M_hat, 4 kernels)",
                       "bytes_per_step": step_bytes,
                       "l2": "inputs larger than L2 (%.2f GB per step vs 0.13 GB L2)" % (step_bytes / 1e9),
                       "parallelism": f"replicas{world}" if world > 1 else "single GPU"},
            "frac_of_peak": round(value / peak, 4),
            "gflops": round(world * 2 * MHAT_FLOP_PER_SITE * vh * args.steps / (ms * 1e-3) / 1e9, 1),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": dom,
                         "kernel_ms": round(dms, 5), "peak_kind": peak_kind},
            "time_to_solution": tts,
            "workload_summary": summarize(extra),
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e, 2), "unit": "GB/s", "h2d_bytes_per_step": vh * 24 * 8,
                    "d2h_bytes_per_step": vh * 24 * 8},
            "gpu_launches": 4 * args.steps,
            "clocks": clocks,
            "tuning": {"even_pass": "staged" if tuning[0] else "direct",
                       "odd_pass": "staged" if tuning[1] else "direct"},
        }
        print(json.dumps(line), flush=True)
    return 0


def summarize(extra):
    """Seconds to solution of each extra workload, a few numbers per workload."""
    out = {}
    ru = extra.get("reliable_update_operator_32x64", {})
    if "double_word_ms" in ru:
        out["reliable_update_op_32x64_ms"] = {"fp64": ru["fp64_ms"], "double_word": ru["double_word_ms"]}
    ms = extra.get("multishift_heavy_24x48", {})
    if "single_refined" in ms:
        out["multishift_24x48_s"] = {k: ms[k]["seconds"] for k in
                                     ("single_refined", "single_half_refined", "half_refined", "double") if k in ms}
    bt = extra.get("batch_uneven_24", {})
    if "batched_s" in bt:
        out["batch_24_s"] = {"batched": bt["batched_s"], "sequential": bt.get("sequential_s")}
    fo = extra.get("force_outer_heavy_24x48", {})
    if "f32_fields" in fo:
        out["force_outer_24x48_frac_of_hbm"] = {k: fo[k]["frac_of_hbm"] for k in ("f32_fields", "f16_fields")}
    ra = extra.get("rational_correction_heavy_24x48", {})
    if "double" in ra:
        out["rational_heatbath_24x48_s"] = {k: ra[k]["heatbath_s"] for k in ("double", "single_single", "single_half")
                                            if k in ra}
    pt = extra.get("ptc_fcg_48x96", {})
    if "ptc_fcg" in pt:
        out["ptc_48x96"] = {"train_pairs": pt.get("train_pairs"), "train_configs": pt.get("train_configs"),
                            "train_s": pt.get("train_s"), "ptc_fcg_s": round(pt["ptc_fcg"]["seconds"], 3),
                            "ptc_fcg_iters": pt["ptc_fcg"]["iters"],
                            "mixed_cg_f16_s": round(pt["mixed_cg_f16"]["seconds"], 3),
                            "fp64_cg_s": round(pt["fp64_cg"]["seconds"], 3)}
    elif "error" in pt:
        out["ptc_48x96"] = {"error": pt["error"][:200]}
    mg = extra.get("mg_gcr_48x96", {})
    if "mg_gcr_s" in mg:
        out["mg_48x96"] = {k: mg[k] for k in ("mg_setup_s", "mg_gcr_s", "mg_gcr_iters", "eo_mixed_cg_s",
                                              "speedup_mg_vs_eo_mixed_cg") if k in mg}
    elif "error" in mg:
        out["mg_48x96"] = {"error": mg["error"][:200]}
    return out


def _sync():
    import torch
    torch.cuda.synchronize()


def run_reliable_update_operator(tm, ctx, bd, dev, reps=10):
    """The operator of the mixed solvers' reliable updates, M_hat^dag M_hat on
    native FP64 fields at the workload's lattice: native FP64 arithmetic
    (tm_apply_Mhat) against double-word arithmetic (tm_apply_Mhat_dw, its
    conversions included), CUDA events, and the relative L2 difference of the
    two results."""
    import torch
    nbytes = tm.tm_field_bytes(ctx, tm.TM_F64, 1)
    a = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    o64 = torch.empty_like(a)
    odw = torch.empty_like(a)
    tm.tm_field_import(ctx, tm.TM_F64, 1, a, bd)
    out = {"op": "M_hat^dag M_hat on native FP64 fields"}
    for name, f in (("fp64_ms", lambda: tm.tm_apply_Mhat(ctx, tm.TM_MDAGM, tm.TM_F64, o64, a)),
                    ("double_word_ms", lambda: tm.tm_apply_Mhat_dw(ctx, tm.TM_MDAGM, odw, a))):
        f()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f()
        e1.record()
        torch.cuda.synchronize()
        out[name] = round(e0.elapsed_time(e1) / reps, 4)
    x = o64.view(torch.float64)
    y = odw.view(torch.float64)
    out["rel_l2_difference"] = float(torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(x))
    out["speedup"] = round(out["fp64_ms"] / out["double_word_ms"], 3)
    return out


def run_multishift(tm, args):
    """Heavy doublet 24^3x48: 12 shifts log-spaced in [1e-5, 1] x the spectral bound of
    Q_h Q_h^dag; multishift CG in the sloppy precision with shift-by-shift
    refinement to 1e-10, against multishift CG in FP64 throughout."""
    import torch
    w = CFG.HEAVY_24
    u = F.gauge_field(w.dims, w.link_seed)
    b = F.odd_spinor(w.dims, w.rhs_seed, 2)
    ctx = tm.tm_create(w.dims, 0)
    out = {"workload": w.name, "lattice": list(w.dims), "mubar": w.mubar, "epsbar": w.epsbar}
    try:
        tm.tm_gauge_load(ctx, u, 1.0)
        tm.tm_clover_compute(ctx, w.kappa, w.csw, mubar=w.mubar, epsbar=w.epsbar, bc_t=w.bc_t)
        for p in (tm.TM_F32, tm.TM_F16):
            tm.tm_autotune(ctx, p, 2)
        t0 = time.perf_counter()
        lam = tm.tm_power_iteration(ctx, tm.TM_QH_SQ, 100)
        out["power_iteration_s"] = round(time.perf_counter() - t0, 4)
        lam_t = 1.02 * lam
        shifts = [lam_t * 10.0 ** (-5 + 5 * k / 11) for k in range(CFG.N_SHIFTS)]
        out["lambda_max"] = lam
        bd = torch.from_numpy(b.view(np.float64).copy()).cuda()
        # (multishift storage, refinement storage): Sec. 4.2's forms "single / double-single",
        # "single / double-half", "half / double-half" and "double"
        forms = (("single_refined", tm.TM_F32, tm.TM_F64), ("single_half_refined", tm.TM_F32, tm.TM_F16),
                 ("half_refined", tm.TM_F16, tm.TM_F64), ("double", tm.TM_F64, tm.TM_F64))
        for name, sl, rf in forms:
            xs = [torch.zeros_like(bd) for _ in shifts]
            _sync()
            t0 = time.perf_counter()
            infos = tm.tm_solve_multishift(ctx, tm.TM_QH_SQ, shifts, xs, bd,
                                           tm.solve_params(tol=w.tol, sloppy=sl, refine=rf), check=False)
            _sync()
            out[name] = {"seconds": round(time.perf_counter() - t0, 4),
                         "max_true_rel_res": max(i.true_rel_res for i in infos),
                         "iters_per_shift": [i.iters for i in infos],
                         "status": sorted({tm.STATUS_NAMES[i.status] for i in infos})}
    finally:
        tm.tm_destroy(ctx)
    return out


def run_batch(tm, args):
    """24 light solves on 8^3x16, 12^3x24, 16^3x32 and 24^3x48 (6 each) advanced
    together by batched kernels, against the same 24 solves one after another."""
    import torch
    ws = CFG.batch_workloads()
    ctxs, bs, xs = [], [], []
    out = {"problems": len(ws), "lattices": sorted({"x".join(map(str, w.dims)) for w in ws})}
    try:
        for w in ws:
            c = tm.tm_create(w.dims, 0)
            ctxs.append(c)
            tm.tm_gauge_load(c, F.gauge_field(w.dims, w.link_seed, workers=1), 1.0)
            tm.tm_clover_compute(c, w.kappa, w.csw, mu=w.mu, bc_t=w.bc_t)
            tm.tm_autotune(c, tm.TM_F16, 1)
            b = F.odd_spinor(w.dims, w.rhs_seed)
            bs.append(torch.from_numpy(b.view(np.float64).copy()).cuda())
            xs.append(torch.zeros_like(bs[-1]))
        sp = tm.solve_params(tol=1e-10, sloppy=tm.TM_F16)
        _sync()
        t0 = time.perf_counter()
        infos = tm.tm_solve_batch(ctxs, tm.TM_MDAGM, sp, xs, bs, check=False)
        _sync()
        out["batched_s"] = round(time.perf_counter() - t0, 4)
        out["batched_max_true_rel_res"] = max(i.true_rel_res for i in infos)
        out["batched_status"] = sorted({tm.STATUS_NAMES[i.status] for i in infos})
        for x in xs:
            x.zero_()
        _sync()
        t0 = time.perf_counter()
        seq = [tm.tm_solve_cg(c, tm.TM_MDAGM, sp, x, b, check=False) for c, x, b in zip(ctxs, xs, bs)]
        _sync()
        out["sequential_s"] = round(time.perf_counter() - t0, 4)
        out["sequential_max_true_rel_res"] = max(i.true_rel_res for i in seq)
        out["speedup_batched_vs_sequential"] = round(out["sequential_s"] / out["batched_s"], 3)
        out["iters"] = [i.iters for i in infos]
    finally:
        for c in ctxs:
            tm.tm_destroy(c)
    return out


def run_force(args, peak):
    """The rational-approximation force step on the heavy doublet at 24^3x48: the
    outer products of 12 two-flavour field pairs (one per shift) on every link,
    one tm_force_outer launch, fields in FP32 and in FP16 storage."""
    from paper_2212_06635_gb300.kernel_timing import force_outer
    dims = CFG.HEAVY_24.dims
    out = {"lattice": list(dims), "pairs": CFG.N_SHIFTS, "flavours": 2,
           "bytes": "2 n V field sites + FP32 links + FP64 force read and written"}
    for name, prec in (("f32_fields", 1), ("f16_fields", 3)):
        ms, b = force_outer(dims, prec, 2, CFG.N_SHIFTS, 20, quiet=True)
        out[name] = {"us_per_launch": round(ms * 1e3, 2), "gb_per_launch": round(b / 1e9, 4),
                     "gbs": round(b / ms / 1e6, 1), "frac_of_hbm": round(b / ms / 1e6 / peak, 4)}
    return out


def run_rational(tm, args):
    """The rational approximation's correction term on the heavy doublet at
    24^3x48 (Fig. 4's table): Zolotarev r(x) ~ x^-1/2 with 12 poles on
    [1e-5, 1] x 1.02 lambda_max; heatbath phi = (1 + Z)^-1/4 eta and acceptance
    <phi, (1 + Z)^1/2 phi>, Z = A r(A)^2 - 1, each rational application one
    multishift solve refined to 1e-10, for the three multishift forms."""
    import torch
    w = CFG.HEAVY_24
    u = F.gauge_field(w.dims, w.link_seed)
    eta = F.odd_spinor(w.dims, w.rhs_seed + 1, 2)
    ctx = tm.tm_create(w.dims, 0)
    out = {"workload": "heavy doublet 24^3x48 rational correction term", "poles": CFG.N_SHIFTS}
    try:
        tm.tm_gauge_load(ctx, u, 1.0)
        tm.tm_clover_compute(ctx, w.kappa, w.csw, mubar=w.mubar, epsbar=w.epsbar, bc_t=w.bc_t)
        for p in (tm.TM_F32, tm.TM_F16):
            tm.tm_autotune(ctx, p, 2)
        lmax = 1.02 * tm.tm_power_iteration(ctx, tm.TM_QH_SQ, 100)
        coeffs = tm.tm_rational_inv_sqrt(CFG.N_SHIFTS, 1e-5 * lmax, lmax)
        out["delta"] = coeffs[3]
        ed = torch.from_numpy(eta.view(np.float64).copy()).cuda()
        ee = float(torch.dot(ed.reshape(-1), ed.reshape(-1)))
        forms = (("double", tm.TM_F64, tm.TM_F64), ("single_single", tm.TM_F32, tm.TM_F64),
                 ("single_half", tm.TM_F32, tm.TM_F16))
        for name, sl, rf in forms:
            sp = tm.solve_params(tol=w.tol, sloppy=sl, refine=rf)
            phi = torch.zeros_like(ed)
            acc = torch.zeros_like(ed)
            _sync()
            t0 = time.perf_counter()
            _, n1 = tm.tm_rational_correction(ctx, tm.TM_QH_SQ, coeffs, -0.25, phi, ed, sp, series_tol=1e-10)
            _sync()
            t1 = time.perf_counter()
            _, n2 = tm.tm_rational_correction(ctx, tm.TM_QH_SQ, coeffs, 0.5, acc, phi, sp, series_tol=1e-10)
            energy = float(torch.dot(phi.reshape(-1), acc.reshape(-1)))
            _sync()
            t2 = time.perf_counter()
            out[name] = {"heatbath_s": round(t1 - t0, 4), "acceptance_s": round(t2 - t1, 4),
                         "z_applications": [n1, n2], "energy_minus_eta2_rel": (energy - ee) / ee}
    finally:
        tm.tm_destroy(ctx)
    return out


def _parity_lex(dims, parity, dev):
    """Lexicographic index of every site of one parity, in the half-lattice order
    of the native fields (site k of that parity has lex // 2 == k)."""
    import torch
    X, Y, Z, T = dims
    lex0 = 2 * torch.arange(X * Y * Z * T // 2, device=dev, dtype=torch.int64)
    r = lex0 // X
    yzt = (r % Y) + ((r // Y) % Z) + (r // (Y * Z))
    return lex0 + ((yzt + parity) % 2)     # x = lex % X: even at lex0, so x parity is the offset


def run_mg(tm, args):
    """48^3x96 (the PTC workload's action): the full system M x = b, b on odd
    sites, to FP64 true relative residual 1e-10 by (a) multigrid-preconditioned
    GCR (Sec. 4.1's method; FP32 hierarchy and inner GCR, FP64 defect correction)
    and (b) the even-odd route of mixed-precision CG: M_hat^dag M_hat y = M_hat^dag b_o
    in FP16 storage, x_o = y, x_e = kappa M_ee^-1 H_eo y.  Both solutions are
    checked by the FP64 full residual; CG's normal-equation tolerance is tightened
    until that residual reaches 1e-10.  Multigrid setup time is reported apart."""
    import torch
    w = CFG.PTC_48
    V = w.volume
    vh = V // 2
    p = CFG.MG_PARAMS
    dev = torch.device("cuda")
    out = {"workload": "full system M x = b at 48^3x96, b on odd sites", "lattice": list(w.dims),
           "mg": {k: (list(v) if isinstance(v, tuple) else v) for k, v in p.items()}}
    ctx = tm.tm_create(w.dims, 0)
    mg = None
    try:
        tm.tm_gauge_load(ctx, F.gauge_field(w.dims, w.link_seed), 1.0)
        tm.tm_clover_compute(ctx, w.kappa, w.csw, mu=w.mu, bc_t=w.bc_t)
        tm.tm_autotune(ctx, tm.TM_F16, 1)
        bod = torch.from_numpy(F.odd_spinor(w.dims, w.rhs_seed).view(np.float64).copy()).to(dev)
        lex_o = _parity_lex(w.dims, 1, dev)
        lex_e = _parity_lex(w.dims, 0, dev)
        bfull = torch.zeros(V, 24, dtype=torch.float64, device=dev)
        bfull[lex_o] = bod.view(vh, 24)
        bfull = bfull.view(-1)
        bn = float(torch.linalg.vector_norm(bfull))

        def full_res(x):
            r = torch.empty_like(bfull)
            tm.tm_apply_full(ctx, 1, tm.TM_F64, r, x)
            torch.cuda.synchronize()
            return float(torch.linalg.vector_norm(bfull - r)) / bn

        # (a) multigrid-preconditioned GCR
        g = torch.Generator(device=dev)
        g.manual_seed(6000)
        init = torch.randn(p["nvec"] * V * 24, dtype=torch.float64, device=dev, generator=g)
        mg = tm.tm_mg_create(ctx, tm.mg_params(p["block"], p["nvec"], p["setup_steps"], p["smooth_steps"], 1,
                                               tm.TM_F32, p["coarse_tol"], p["coarse_maxiter"], p["coarse_restart"]))
        _sync()
        t0 = time.perf_counter()
        tm.tm_mg_setup(mg, init)
        _sync()
        out["mg_setup_s"] = round(time.perf_counter() - t0, 3)
        del init
        x = torch.zeros_like(bfull)
        info = tm.tm_solve_gcr(ctx, 1, mg, tm.solve_params(tol=w.tol, maxiter=p["maxiter"], sloppy=tm.TM_F32,
                                                           chunk=p["restart"]), x, bfull, check=False)
        out["mg_gcr"] = info.as_dict()
        out["mg_gcr_s"] = round(info.seconds, 3)
        out["mg_gcr_iters"] = info.iters
        out["mg_gcr_full_res"] = full_res(x)
        tm.tm_mg_destroy(mg)
        mg = None
        # (b) even-odd mixed CG on the normal equations
        g5b = bod.view(vh, 4, 6).clone()
        g5b[:, 2:, :] *= -1.0
        nb64 = tm.tm_field_bytes(ctx, tm.TM_F64, 1)
        fa = torch.empty(nb64, dtype=torch.uint8, device=dev)
        fb = torch.empty(nb64, dtype=torch.uint8, device=dev)
        c = torch.empty_like(bod)
        tm.tm_field_import(ctx, tm.TM_F64, 1, fa, g5b.view(-1))
        tm.tm_apply_Mhat(ctx, tm.TM_QHAT_MINUS, tm.TM_F64, fb, fa)     # M_hat^dag b_o = Q_hat_- g5 b_o
        tm.tm_field_export(ctx, tm.TM_F64, 1, c, fb)
        y = torch.zeros_like(bod)
        xe = torch.empty_like(bod)
        for tol in (1e-10, 1e-11, 1e-12):
            y.zero_()
            inf = tm.tm_solve_cg(ctx, tm.TM_MDAGM, tm.solve_params(tol=tol, sloppy=tm.TM_F16), y, c, check=False)
            t0 = time.perf_counter()
            tm.tm_field_import(ctx, tm.TM_F64, 1, fa, y)
            tm.tm_apply_even(ctx, tm.TM_QHAT_PLUS, tm.TM_F64, fb, fa)
            tm.tm_field_export(ctx, tm.TM_F64, 1, xe, fb)
            xf = torch.empty(V, 24, dtype=torch.float64, device=dev)
            xf[lex_o] = y.view(vh, 24)
            xf[lex_e] = w.kappa * xe.view(vh, 24)
            _sync()
            recon = time.perf_counter() - t0
            res = full_res(xf.view(-1))
            out["eo_mixed_cg"] = {"normal_tol": tol, "iters": inf.iters, "seconds": round(inf.seconds + recon, 3),
                                  "full_res": res, "status": tm.STATUS_NAMES[inf.status]}
            if res <= w.tol:
                break
        out["eo_mixed_cg_s"] = out["eo_mixed_cg"]["seconds"]
        out["speedup_mg_vs_eo_mixed_cg"] = round(out["eo_mixed_cg_s"] / max(out["mg_gcr_s"], 1e-9), 3)
    finally:
        if mg is not None:
            tm.tm_mg_destroy(mg)
        tm.tm_destroy(ctx)
    return out


def run_ptc(tm, args):
    """48^3x96: train the 4-layer 8-channel PTC network on solver-generated pairs
    from several seeded configurations, then solve on the benchmark configuration
    with PTC-preconditioned flexible CG vs mixed-precision CG vs FP64 CG."""
    import torch
    w = CFG.PTC_48
    out = {"workload": w.name, "lattice": list(w.dims), "channels": [1, 8, 8, 8, 1]}
    net = tm.tm_ptc_create([1, 8, 8, 8, 1])
    ctxs = []
    try:
        tm.tm_ptc_init(net, scale=0.5, noise=0.02, seed=4000)
        # one configuration resident at a time (a 48^3x96 context holds ~45 GB);
        # the Adam state lives in the network, so training continues across them
        per = max(1, args.ptc_pairs // args.ptc_configs)
        setup_s, train_s, losses = 0.0, 0.0, []
        for j in range(args.ptc_configs):
            t0 = time.perf_counter()
            c = tm.tm_create(w.dims, 0)
            ctxs.append(c)
            tm.tm_gauge_load(c, F.gauge_field(w.dims, 4000 + j), 1.0)
            tm.tm_clover_compute(c, w.kappa, w.csw, mu=w.mu, bc_t=w.bc_t)
            _sync()
            t1 = time.perf_counter()
            losses.append(tm.tm_ptc_train(net, [c], tm.TM_MDAGM, npairs=per, batch=8, lr=2e-3, seed=5000 + 1000 * j))
            _sync()
            t2 = time.perf_counter()
            setup_s += t1 - t0
            train_s += t2 - t1
            tm.tm_destroy(c)
            ctxs.pop()
        losses = np.concatenate(losses)
        out["config_setup_s"] = round(setup_s, 2)
        out["train_s"] = round(train_s, 2)
        out["train_pairs"] = int(len(losses))
        out["train_configs"] = args.ptc_configs
        out["loss_first64"] = float(np.mean(losses[:64]))
        out["loss_last64"] = float(np.mean(losses[-64:]))
        c = tm.tm_create(w.dims, 0)
        ctxs.append(c)
        tm.tm_gauge_load(c, F.gauge_field(w.dims, w.link_seed), 1.0)
        tm.tm_clover_compute(c, w.kappa, w.csw, mu=w.mu, bc_t=w.bc_t)
        tm.tm_autotune(c, tm.TM_F16, 1)
        b = F.odd_spinor(w.dims, w.rhs_seed)
        bd = torch.from_numpy(b.view(np.float64).copy()).cuda()
        x = torch.zeros_like(bd)
        info = tm.tm_solve_fcg(c, tm.TM_MDAGM, net, tm.solve_params(tol=w.tol), x, bd, check=False)
        out["ptc_fcg"] = info.as_dict()
        for name, sl in (("mixed_cg_f16", tm.TM_F16), ("fp64_cg", tm.TM_F64)):
            x.zero_()
            inf = tm.tm_solve_cg(c, tm.TM_MDAGM, tm.solve_params(tol=w.tol, sloppy=sl), x, bd, check=False)
            out[name] = inf.as_dict()
        out["speedup_ptc_fcg_vs_fp64_cg"] = round(out["fp64_cg"]["seconds"] / out["ptc_fcg"]["seconds"], 3)
        out["speedup_ptc_fcg_vs_mixed_cg"] = round(out["mixed_cg_f16"]["seconds"] / out["ptc_fcg"]["seconds"], 3)
    finally:
        tm.tm_ptc_destroy(net)
        for c in ctxs:
            tm.tm_destroy(c)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f16", choices=["f16", "bf16", "f32"])
    ap.add_argument("--variant", default="auto", choices=["auto", "direct", "staged"],
                    help="stencil variant of the step (auto: the autotuner's choice)")
    ap.add_argument("--maxiter", type=int, default=60000)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 CG time-to-solution leg")
    ap.add_argument("--no-solve", action="store_true", help="skip both time-to-solution legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the heavy multishift and uneven batch workloads")
    ap.add_argument("--no-ptc", action="store_true",
                    help="skip the PTC training + PTC-FCG workload on 48^3x96")
    ap.add_argument("--no-mg", action="store_true", help="skip the multigrid workload on 48^3x96")
    ap.add_argument("--ptc-quick", action="store_true",
                    help="short PTC training (512 pairs from 2 configurations) instead of the workload's "
                         "2048 pairs from 8 configurations")
    ap.add_argument("--ptc-pairs", type=int, default=None)
    ap.add_argument("--ptc-configs", type=int, default=None)
    args = ap.parse_args()
    if args.ptc_pairs is None:
        args.ptc_pairs = 512 if args.ptc_quick else 2048
    if args.ptc_configs is None:
        args.ptc_configs = 2 if args.ptc_quick else 8
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
