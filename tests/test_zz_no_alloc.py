"""tm_field_norm2_noalloc: the squared norm for callers that cannot allocate
device memory when they need one (a host framework whose pool owns the whole
device memory budget, or a latency-critical loop that must never reach the
allocator, whose cudaMalloc / cudaFree can synchronise the device).

It must give the same result as tm_field_norm2 and as an independent long-double
sum of the stored field on the host, on two calls in a row (the shared scratch
array keeps the previous call's contents, so the second call checks that nothing
stale leaks in); it must refuse fields larger than its fixed scratch array and
pointers that are not device memory.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from synth import fields as F

pytestmark = pytest.mark.gpu

TOL = 1e-13   # relative; both entry points run the same deterministic reduction


def _host_tol(prec, nf):
    """Bound of the reduction against an exact sum of the stored values: FP64
    arithmetic is exact to about 1e-13 here; FP32 and 16-bit fields sum each
    site's 2 * 12 nf squares in FP32 (one rounding per square and per addition,
    plus one for the 16-bit scale), then in FP64 across sites."""
    if prec == 0:
        return 1e-13
    return (2 * 2 * 12 * nf + 2) * 2.0 ** -24


def _field(tm, ctx, prec, nf, dims, seed):
    import torch
    b = F.odd_spinor(dims, seed, nf)
    src = torch.from_numpy(b.view(np.float64).copy()).cuda()
    f = torch.empty(tm.tm_field_bytes(ctx, prec, nf), dtype=torch.uint8, device="cuda")
    tm.tm_field_import(ctx, prec, nf, f, src)
    return f, src


def _host_norm2(tm, ctx, prec, nf, f, like):
    """||f||^2 of the stored (de-quantised) field, summed on the host in long double."""
    import torch
    out = torch.empty_like(like)
    tm.tm_field_export(ctx, prec, nf, out, f)
    torch.cuda.synchronize()
    x = out.cpu().numpy().astype(np.longdouble)
    return float(np.sum(x * x))


@pytest.mark.parametrize("prec,nf", [(0, 1), (3, 1), (1, 2), (2, 2)], ids=["f64", "f16", "f32-heavy", "bf16-heavy"])
def test_noalloc_norm_matches_allocating_norm(prec, nf):
    import torch
    from paper_2212_06635_gb300 import tm
    dims = (8, 6, 4, 10)
    ctx = tm.tm_create(dims, 0)
    try:
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        for call, seed in enumerate((71, 72)):       # two calls in a row, different data
            f, src = _field(tm, ctx, prec, nf, dims, seed)
            tm.tm_field_norm2(ctx, prec, nf, f, out[0:1])
            tm.tm_field_norm2_noalloc(ctx, prec, nf, f, out[1:2])
            torch.cuda.synchronize()
            ref, got = float(out[0]), float(out[1])
            assert ref > 0
            assert abs(got - ref) <= TOL * ref, (call, got, ref)
            host = _host_norm2(tm, ctx, prec, nf, f, src)
            assert abs(got - host) <= _host_tol(prec, nf) * host, (call, got, host)
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


def test_noalloc_rejects_host_pointers():
    """A host address for the result or the field is refused before any launch
    (the kernel would otherwise write through it on the GPU)."""
    import torch
    from paper_2212_06635_gb300 import tm
    dims = (4, 4, 4, 4)
    ctx = tm.tm_create(dims, 0)
    try:
        f, _ = _field(tm, ctx, tm.TM_F64, 1, dims, 73)
        host_out = np.zeros(2, dtype=np.float64)
        with pytest.raises(tm.TMError) as e:
            tm.tm_field_norm2_noalloc(ctx, tm.TM_F64, 1, f, host_out)
        assert e.value.status == tm.TM_ERR_ARG
        assert "device pointers" in tm.tm_last_error()
        host_field = np.zeros(f.numel() // 8 + 2, dtype=np.float64)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(tm.TMError) as e:
            tm.tm_field_norm2_noalloc(ctx, tm.TM_F64, 1, host_field, out)
        assert e.value.status == tm.TM_ERR_ARG
        # the context and the entry point stay usable
        tm.tm_field_norm2_noalloc(ctx, tm.TM_F64, 1, f, out)
        torch.cuda.synchronize()
        assert float(out[0]) > 0
    finally:
        tm.tm_destroy(ctx)
