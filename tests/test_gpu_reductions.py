"""Reductions against an independent host sum (pin P13 of the hot-path table):
tm_field_norm2 of a stored field equals the long-double sum of the squares of
the same stored values, exported to the host.

The check runs at 32^3x64 (1,048,576 odd sites: 4096 blocks of 256 threads, many
waves on 152 SMs, so the two-level block reduction and its last-block
finalisation are exercised) and at a ragged lattice whose last block is partly
empty, in every storage precision, light and heavy.  Bound: FP64 fields sum in
FP64 (1e-13 relative over a million terms); FP32 and 16-bit fields sum each
site's 2 * 12 nf squares in FP32 (one rounding per square and per addition, and
one for the 16-bit scale) before the FP64 reduction across sites.
"""
import numpy as np
import pytest

from synth import fields as F

pytestmark = pytest.mark.gpu


def _tol(prec, nf):
    if prec == 0:
        return 1e-13
    return (2 * 2 * 12 * nf + 2) * 2.0 ** -24


@pytest.fixture(scope="module")
def ctx32():
    from paper_2212_06635_gb300 import tm
    ctx = tm.tm_create((32, 32, 32, 64), 0)
    yield tm, ctx
    tm.tm_destroy(ctx)


def _check(tm, ctx, dims, prec, nf, seed):
    import torch
    b = F.odd_spinor(dims, seed, nf)
    src = torch.from_numpy(b.view(np.float64).copy()).cuda()
    f = torch.empty(tm.tm_field_bytes(ctx, prec, nf), dtype=torch.uint8, device="cuda")
    tm.tm_field_import(ctx, prec, nf, f, src)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    tm.tm_field_norm2(ctx, prec, nf, f, out)
    back = torch.empty_like(src)
    tm.tm_field_export(ctx, prec, nf, back, f)
    torch.cuda.synchronize()
    x = back.cpu().numpy().astype(np.longdouble)
    host = float(np.sum(x * x))
    got = float(out[0])
    assert host > 0
    assert abs(got - host) <= _tol(prec, nf) * host, (prec, nf, got, host, abs(got - host) / host)
    # the stored field is the imported one up to its storage rounding
    exact = float(np.sum(b.view(np.float64).astype(np.longdouble) ** 2))
    assert abs(host - exact) <= (1e-15 if prec == 0 else 2e-2) * exact


@pytest.mark.parametrize("prec", [0, 1, 3, 2], ids=["f64", "f32", "f16", "bf16"])
def test_norm2_vs_host_long_double_32x64(ctx32, prec):
    tm, ctx = ctx32
    _check(tm, ctx, (32, 32, 32, 64), prec, 1, 2101 + prec)


@pytest.mark.parametrize("prec", [0, 1, 3, 2], ids=["f64", "f32", "f16", "bf16"])
def test_norm2_vs_host_long_double_heavy_ragged(prec):
    from paper_2212_06635_gb300 import tm
    dims = (10, 6, 6, 14)                  # 2520 odd sites: 9 full blocks and a ragged tail
    ctx = tm.tm_create(dims, 0)
    try:
        _check(tm, ctx, dims, prec, 2, 2111 + prec)
        _check(tm, ctx, dims, prec, 1, 2121 + prec)
    finally:
        tm.tm_destroy(ctx)
