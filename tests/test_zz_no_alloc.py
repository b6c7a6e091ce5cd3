"""tm_field_norm2_noalloc: the squared norm for callers that may not allocate
device memory at call time (for example during CUDA-graph stream capture, or in
a loop that must never reach the allocator).  It must give the same result as
tm_field_norm2, on two calls in a row (the shared scratch array keeps the
previous call's contents, so the second call checks that nothing stale leaks
in), and must refuse fields larger than its fixed scratch array.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from synth import fields as F

pytestmark = pytest.mark.gpu

TOL = 1e-13   # relative; both entry points run the same deterministic reduction


def _field(tm, ctx, prec, nf, dims, seed):
    import torch
    b = F.odd_spinor(dims, seed, nf)
    src = torch.from_numpy(b.view(np.float64).copy()).cuda()
    f = torch.empty(tm.tm_field_bytes(ctx, prec, nf), dtype=torch.uint8, device="cuda")
    tm.tm_field_import(ctx, prec, nf, f, src)
    return f


@pytest.mark.parametrize("prec,nf", [(0, 1), (3, 1), (1, 2), (2, 2)], ids=["f64", "f16", "f32-heavy", "bf16-heavy"])
def test_noalloc_norm_matches_allocating_norm(prec, nf):
    import torch
    from paper_2212_06635_gb300 import tm
    dims = (8, 6, 4, 10)
    ctx = tm.tm_create(dims, 0)
    try:
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        for call, seed in enumerate((71, 72)):       # two calls in a row, different data
            f = _field(tm, ctx, prec, nf, dims, seed)
            tm.tm_field_norm2(ctx, prec, nf, f, out[0:1])
            tm.tm_field_norm2_noalloc(ctx, prec, nf, f, out[1:2])
            torch.cuda.synchronize()
            ref, got = float(out[0]), float(out[1])
            assert ref > 0
            assert abs(got - ref) <= TOL * ref, (call, got, ref)
    finally:
        tm.tm_destroy(ctx)


def test_noalloc_rejects_fields_beyond_the_scratch_array():
    import torch
    from paper_2212_06635_gb300 import tm
    ctx = tm.tm_create((64, 64, 64, 130), 0)    # 17,039,360 sites per parity
    try:
        f = torch.zeros(16, dtype=torch.uint8, device="cuda")
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(tm.TMError) as e:
            tm.tm_field_norm2_noalloc(ctx, tm.TM_F64, 1, f, out)
        assert e.value.status == tm.TM_ERR_ARG
        assert "too large" in tm.tm_last_error()
    finally:
        tm.tm_destroy(ctx)
