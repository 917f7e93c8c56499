"""torch.autograd.Function for C = A·B on the library's kernels.

Forward: C = A·B (row-major tensors).  Backward: dA = dC·B^T and dB = A^T·dC, both
computed by the same column-major product with the transposed-operand forms
(Section 8 of the paper: transposed products "on the same footing"), so no
transpose is ever materialised.

BF16 inputs run on the tcgen05 tensor cores with FP32 accumulation (output BF16 by
default, or FP32); FP64 inputs run on the native FP64 kernel, or on the
FP64-accurate slice form when ``compute=COMPUTE_64F_OZAKI``.
"""
from __future__ import annotations

import torch

from . import hsmm as _h


def _mm(a, b, trans_a=False, trans_b=False, out_dtype=None, compute=None):
    kw = {}
    if a.dtype == torch.float64:
        kw["compute"] = _h.COMPUTE_64F_NATIVE if compute is None else compute
    return _h.matmul(a, b, trans_a=trans_a, trans_b=trans_b, out_dtype=out_dtype, **kw)


class HsmmMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a: torch.Tensor, b: torch.Tensor, out_dtype=None, compute=None):
        if a.dim() != 2 or b.dim() != 2 or a.shape[1] != b.shape[0]:
            raise ValueError(f"shapes {tuple(a.shape)} x {tuple(b.shape)} do not multiply")
        if a.dtype != b.dtype or a.dtype not in (torch.bfloat16, torch.float64):
            raise TypeError("HsmmMatmul takes two BF16 or two FP64 tensors")
        a = a.contiguous()
        b = b.contiguous()
        ctx.save_for_backward(a, b)
        ctx.compute = compute
        dt = out_dtype if out_dtype is not None else a.dtype
        return _mm(a, b, out_dtype=dt, compute=compute)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        a, b = ctx.saved_tensors
        g = g.contiguous()
        if g.dtype != a.dtype:
            g = g.to(a.dtype)
        da = db = None
        if ctx.needs_input_grad[0]:
            da = _mm(g, b, trans_b=True, out_dtype=a.dtype, compute=ctx.compute)     # dC · B^T
        if ctx.needs_input_grad[1]:
            db = _mm(a, g, trans_a=True, out_dtype=b.dtype, compute=ctx.compute)     # A^T · dC
        return da, db, None, None


def hsmm_matmul(a: torch.Tensor, b: torch.Tensor, out_dtype=None, compute=None) -> torch.Tensor:
    return HsmmMatmul.apply(a, b, out_dtype, compute)
