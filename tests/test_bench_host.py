"""Host-side logic of bench.py: the max-over-ranks timing and whole-job
aggregation of the replicated (weak-scaling) multi-GPU run, exercised with two
gloo ranks on the CPU, and the reference arm (the CPU oracle) JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 1.0 + rank          # rank 1 is the slow one
    m = bench.max_over_ranks(local)
    q.put((rank, m, bench.aggregate_gbs(world, 2.0e9, 10, m)))
    tdist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, gbs in res:
        assert m == 2.0                         # the slowest rank's time
        assert abs(gbs - 2 * 2.0e9 * 10 / 2.0 / 1e9) < 1e-9


def test_single_process_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GB/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_parity_lex_matches_the_half_lattice_order():
    """The bench embeds odd-site fields into full canonical fields with
    _parity_lex: site k of a parity must be the k-th site of that parity in
    lexicographic order (the native half-lattice order, lex // 2 == k)."""
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    from oracle import dirac as D
    for dims in ((4, 4, 4, 4), (6, 4, 2, 8), (2, 6, 4, 2)):
        geo = D.Geometry(dims)
        for parity, ref in ((0, geo.even), (1, geo.odd)):
            got = bench._parity_lex(dims, parity, torch.device("cpu")).numpy()
            assert np.array_equal(got, ref), (dims, parity)


def test_workload_summary_keeps_the_times():
    sys.path.insert(0, ROOT)
    import bench
    extra = {"batch_uneven_24": {"batched_s": 0.48, "sequential_s": 0.59},
             "mg_gcr_48x96": {"mg_setup_s": 5.9, "mg_gcr_s": 28.9, "mg_gcr_iters": 381, "eo_mixed_cg_s": 1.08,
                              "speedup_mg_vs_eo_mixed_cg": 0.037, "mg_gcr": {"iters": 381}},
             "ptc_fcg_48x96": {"error": "RuntimeError('x')"},
             "reliable_update_operator_32x64": {"fp64_ms": 9.8, "double_word_ms": 3.7, "speedup": 2.65,
                                                "rel_l2_difference": 6e-15}}
    out = bench.summarize(extra)
    assert out["reliable_update_op_32x64_ms"] == {"fp64": 9.8, "double_word": 3.7}
    assert out["batch_24_s"] == {"batched": 0.48, "sequential": 0.59}
    assert out["mg_48x96"]["mg_gcr_iters"] == 381 and "mg_gcr" not in out["mg_48x96"]
    assert out["ptc_48x96"]["error"].startswith("RuntimeError")
