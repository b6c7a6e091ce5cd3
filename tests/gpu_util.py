"""Shared helpers of the GPU parity tests: move canonical complex128 fields
between numpy and the device, and drive the C ABI through the binding."""
import numpy as np

# relative L2 error vs the FP64 oracle of one operator application: 1e-13 FP64,
# 1e-6 FP32, 3e-3 16-bit storage.  FP16 (11-bit significand) holds 3e-3 for the
# normal operators too (measured about 5e-4).  BF16 has an 8-bit significand: one
# stored BF16 field alone carries about 2e-3 relative error, so a normal operator
# (two applications with a stored BF16 intermediate) gets twice the bound.
PREC_TOL = {0: 1e-13, 1: 1e-6, 2: 3e-3, 3: 3e-3}
# double-word arithmetic (tm_apply_Mhat_dw): unit roundoff 2^-47 of the double-word
# sum, the input and output rounded to 48 bits, a few hundred operations per
# output element over the two passes of a Schur operator: 1e-13 per application,
# 2e-13 for a normal operator
DW_TOL = 1e-13


def tol(prec, napply=1):
    return PREC_TOL[prec] * (napply if prec == 2 else 1)


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def to_dev(a):
    torch, dev = torch_dev()
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)


def from_dev(t, shape):
    return t.detach().cpu().numpy().view(np.complex128).reshape(shape)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


class Lat:
    """A context with a gauge field and clover term loaded."""

    def __init__(self, u, dims, kappa, csw, mu=0.0, mubar=0.0, epsbar=0.0, bc_t=-1, gauge_id=1.0, rho=0.0):
        from paper_2212_06635_gb300 import tm
        self.tm = tm
        self.dims = dims
        self.vh = int(np.prod(dims)) // 2
        self.ctx = tm.tm_create(dims, 0)
        tm.tm_gauge_load(self.ctx, np.ascontiguousarray(u), gauge_id)
        tm.tm_clover_compute(self.ctx, kappa, csw, mu=mu, mubar=mubar, epsbar=epsbar, bc_t=bc_t, rho=rho)

    def close(self):
        if self.ctx:
            self.tm.tm_destroy(self.ctx)
            self.ctx = None

    def native(self, prec, nf):
        torch, dev = torch_dev()
        return torch.empty(self.tm.tm_field_bytes(self.ctx, prec, nf), dtype=torch.uint8, device=dev)

    def apply(self, op, prec, psi):
        """op applied to a canonical odd field through import -> apply -> export."""
        nf = 1 if psi.ndim == 3 else 2
        src = to_dev(psi)
        a = self.native(prec, nf)
        o = self.native(prec, nf)
        self.tm.tm_field_import(self.ctx, prec, nf, a, src)
        self.tm.tm_apply_Mhat(self.ctx, op, prec, o, a)
        out = src.clone()
        self.tm.tm_field_export(self.ctx, prec, nf, out, o)
        import torch
        torch.cuda.synchronize()
        return from_dev(out, psi.shape)

    def apply_dw(self, op, psi):
        """op applied in double-word arithmetic (tm_apply_Mhat_dw) on FP64 fields."""
        nf = 1 if psi.ndim == 3 else 2
        src = to_dev(psi)
        a = self.native(0, nf)
        o = self.native(0, nf)
        self.tm.tm_field_import(self.ctx, 0, nf, a, src)
        self.tm.tm_apply_Mhat_dw(self.ctx, op, o, a)
        out = src.clone()
        self.tm.tm_field_export(self.ctx, 0, nf, out, o)
        import torch
        torch.cuda.synchronize()
        return from_dev(out, psi.shape)
