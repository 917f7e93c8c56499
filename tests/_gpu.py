"""Helpers of the GPU parity tests: column-major device copies of seeded host inputs."""
import numpy as np
import pytest
import torch

import workloads as W

requires_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def hsmm():
    import paper_cs_9809105_gb300 as h
    h.lib()      # raises if the extension is missing: no fallback
    return h


def dev_colmajor(X: np.ndarray, dtype=None, ld=None, device="cuda"):
    """Column-major device copy of a host matrix (optionally with a padded leading dimension)."""
    rows, cols = X.shape
    ld = rows if ld is None else ld
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(X).T))
    if dtype is not None:
        t = t.to(dtype)
    base = torch.zeros((max(cols, 1), max(ld, 1)), dtype=t.dtype, device=device)
    base[:cols, :rows] = t.to(device)
    return base.t()[:rows, :cols]


def dev_bf16_colmajor(bits: np.ndarray, ld=None, device="cuda"):
    """Column-major BF16 device matrix from 16-bit patterns."""
    rows, cols = bits.shape
    ld = rows if ld is None else ld
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(bits, dtype=np.uint16).T).view(np.int16))
    base = torch.zeros((max(cols, 1), max(ld, 1)), dtype=torch.int16, device=device)
    base[:cols, :rows] = t.to(device)
    return base.view(torch.bfloat16).t()[:rows, :cols]


def host(x: torch.Tensor) -> np.ndarray:
    """Host float64 (or integer) copy of a device matrix, column-major order preserved as values."""
    if x.dtype == torch.bfloat16:
        x = x.float()
    return np.asfortranarray(x.cpu().numpy().astype(np.float64 if x.is_floating_point() else np.int64))


def padded(rows, mult=8):
    return W.pad_ld(rows, mult)
