"""torch.autograd.Function over the mixed-distribution NLL kernels.

L = -log(w0 p_tilde(t*) + w1 p_ng(t*)), w = softmax(theta),
p_tilde = softmax(z / tau + b)  (the adaptive head of Sec. 3.6 mixed as in
Sec. 3.5).  Forward and backward run in libnc24's CUDA kernels
(nc_mix_nll_fwd / nc_mix_nll_bwd); gradients flow to b and theta only.
"""
from __future__ import annotations

import torch

from . import nc24


class MixedNLL(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, theta, z, p_ng, target, warm, tau: float = 1.0):
        for t in (b, theta, z, p_ng):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("MixedNLL expects contiguous float32 CUDA tensors")
        target = target.to(torch.int32).contiguous()
        warm = warm.to(torch.int32).contiguous()
        loss = torch.empty(z.shape[0], device=z.device, dtype=torch.float32)
        st = nc24.nc_mix_nll_fwd(z, b, p_ng, theta, target, warm, tau, loss)
        if st:
            raise nc24.NcError(st, "nc_mix_nll_fwd")
        ctx.save_for_backward(b, theta, z, p_ng, target, warm)
        ctx.tau = tau
        return loss

    @staticmethod
    def backward(ctx, gout):
        b, theta, z, p_ng, target, warm = ctx.saved_tensors
        gout = gout.to(torch.float32).contiguous()
        db = torch.empty_like(b)
        dth = torch.empty_like(theta)
        st = nc24.nc_mix_nll_bwd(z, b, p_ng, theta, target, warm, gout, ctx.tau, db, dth)
        if st:
            raise nc24.NcError(st, "nc_mix_nll_bwd")
        return db, dth, None, None, None, None, None


def mixed_nll(b, theta, z, p_ng, target, warm, tau: float = 1.0):
    return MixedNLL.apply(b, theta, z, p_ng, target, warm, tau)
