"""hsmm: GB300-native dense products after "Hyper-Systolic Matrix Multiplication".

The compute path is libhsmm.so (hand-written CUDA for sm_103a, C ABI in
include/hsmm.h); this package is its Python binding plus a torch.autograd
Function and the grouped-launch helpers.
"""
from .hsmm import (C_64F, COMPUTE_32F_FAST_TF32, COMPUTE_64F_NATIVE, COMPUTE_64F_OZAKI, COMPUTE_64F_RING,
                   COMPUTE_DEFAULT, R_8I, R_16BF, R_32F, R_32I, R_64F, GroupedPlan, HsmmError, colmajor, gemm,
                   gemm_grouped, gemm_grouped_workspace_size, gemm_host, gemv, nbody, launch_count,
                   lib, matmul, ozaki_split, ring_gemm, selftest_timeout, set_wait_timeout_ns, sync_status,
                   to_colmajor, workspace_size)

__all__ = ["gemm", "gemm_grouped", "gemm_grouped_workspace_size", "gemm_host", "gemv", "nbody", "matmul", "ring_gemm", "ozaki_split", "GroupedPlan", "colmajor", "to_colmajor", "lib",
           "sync_status", "selftest_timeout", "set_wait_timeout_ns", "launch_count", "workspace_size", "HsmmError",
           "R_64F", "C_64F", "R_32F", "R_16BF", "R_8I", "R_32I", "COMPUTE_DEFAULT", "COMPUTE_32F_FAST_TF32",
           "COMPUTE_64F_NATIVE", "COMPUTE_64F_OZAKI", "COMPUTE_64F_RING"]
