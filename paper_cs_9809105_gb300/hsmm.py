"""ctypes binding of libhsmm (the C ABI declared in include/hsmm.h).

Argument marshalling only: every step of every product runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  If the compiled
library is missing, importing the functions raises -- there is no fallback.

Matrices passed to the column-major calls are torch CUDA tensors whose first
index is contiguous (``stride(0) == 1``); ``colmajor()`` makes one.  Row-major
PyTorch matrices go through ``matmul()``, which maps C = op(A) op(B) onto the
column-major product C^T = op(B)^T op(A)^T without copies.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhsmm.so")

# status codes (hsmm_status_t)
SUCCESS, INVALID_VALUE, NOT_SUPPORTED, WORKSPACE_TOO_SMALL, CUDA_ERROR, TIMEOUT = range(6)
# dtypes (hsmm_dtype_t)
R_64F, R_32F, R_16BF, R_8I, R_32I, C_64F = range(6)
# compute modes (hsmm_compute_t)
COMPUTE_DEFAULT, COMPUTE_32F_FAST_TF32, COMPUTE_64F_NATIVE, COMPUTE_64F_OZAKI, COMPUTE_64F_RING = range(5)

_TORCH2H = {torch.float64: R_64F, torch.float32: R_32F, torch.bfloat16: R_16BF, torch.int8: R_8I,
            torch.int32: R_32I, torch.complex128: C_64F}


class HsmmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({last_error_detail()})")


class Config(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int), ("b", ctypes.c_int), ("c", ctypes.c_int), ("compute", ctypes.c_int),
                ("ozaki_slices", ctypes.c_int), ("ozaki_bits", ctypes.c_int), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("tile_n", ctypes.c_int), ("ring_p", ctypes.c_int), ("ring_k", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


class GemmDesc(ctypes.Structure):
    _fields_ = [("transA", ctypes.c_int), ("transB", ctypes.c_int), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("k", ctypes.c_int64), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64), ("ldc", ctypes.c_int64)]


EXPORTS = ("hsmm_gemm", "hsmm_gemm_host", "hsmm_gemm_host_workspace_size", "hsmm_nbody", "hsmm_gemv", "hsmm_gemv_n_noalloc", "hsmm_gemm_grouped", "hsmm_gemm_grouped_workspace_size", "hsmm_grouped_plan_create", "hsmm_grouped_plan_create_ex", "hsmm_grouped_plan_launch",
           "hsmm_grouped_plan_info", "hsmm_grouped_plan_destroy", "hsmm_ring_gemm", "hsmm_ring_workspace_size", "hsmm_ozaki_split", "hsmm_ozaki_slice_products", "hsmm_ozaki_recombine",
           "hsmm_workspace_size", "hsmm_gemv_workspace_size", "hsmm_sync_status", "hsmm_set_wait_timeout_ns",
           "hsmm_selftest_timeout", "hsmm_status_string", "hsmm_last_cuda_error", "hsmm_last_error_detail", "hsmm_version",
           "hsmm_launch_count")

_lib = None


def lib():
    """Load libhsmm.so (built by __graft_entry__.build() or paper_cs_9809105_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhsmm.so is not built ({LIB_PATH}); run paper_cs_9809105_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    i64, vp, ci, sz = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    P = ctypes.POINTER
    L.hsmm_gemm.argtypes = [P(Config), ci, ci, i64, i64, i64, vp, vp, i64, vp, i64, vp, vp, i64, vp]
    L.hsmm_gemm_host.argtypes = [P(Config), ci, ci, i64, i64, i64, vp, vp, i64, vp, i64, vp, vp, i64, vp]
    L.hsmm_gemm_host_workspace_size.argtypes = [P(Config), ci, ci, i64, i64, i64, P(sz)]
    L.hsmm_nbody.argtypes = [i64, i64, vp, vp, ctypes.c_float, vp, ci, ci, vp]
    L.hsmm_gemv.argtypes = [P(Config), ci, i64, i64, vp, vp, i64, vp, i64, vp, vp, i64, vp]
    L.hsmm_gemm_grouped.argtypes = [P(Config), i64, P(GemmDesc), vp, vp, vp]
    L.hsmm_gemm_grouped_workspace_size.argtypes = [P(Config), i64, P(GemmDesc), P(sz)]
    L.hsmm_gemv_n_noalloc.argtypes = [ci, i64, i64, vp, vp, i64, vp, i64, vp, vp, i64, vp]
    L.hsmm_grouped_plan_create.argtypes = [P(Config), i64, P(GemmDesc), P(vp)]
    L.hsmm_grouped_plan_create_ex.argtypes = [P(Config), i64, P(GemmDesc), P(ci), ci, P(vp)]
    L.hsmm_grouped_plan_launch.argtypes = [vp, vp, vp, vp]
    L.hsmm_grouped_plan_info.argtypes = [vp, P(i64), P(ci)]
    L.hsmm_grouped_plan_destroy.argtypes = [vp]
    L.hsmm_ring_gemm.argtypes = [ci, ci, i64, vp, i64, vp, i64, vp, i64, vp, sz, vp]
    L.hsmm_ring_workspace_size.argtypes = [ci, ci, i64, P(sz)]
    L.hsmm_ozaki_split.argtypes = [i64, i64, vp, i64, ci, ci, ci, vp, vp, i64, i64, vp]
    L.hsmm_ozaki_slice_products.argtypes = [i64, i64, i64, ci, ci, vp, i64, vp, i64, i64, vp, i64, vp]
    L.hsmm_ozaki_recombine.argtypes = [i64, i64, ci, ci, vp, i64, vp, vp, vp, vp, vp, i64, vp]
    L.hsmm_workspace_size.argtypes = [P(Config), ci, ci, i64, i64, i64, P(sz)]
    L.hsmm_gemv_workspace_size.argtypes = [P(Config), ci, i64, i64, P(sz)]
    L.hsmm_sync_status.argtypes = [vp]
    L.hsmm_set_wait_timeout_ns.argtypes = [ctypes.c_uint64]
    L.hsmm_selftest_timeout.argtypes = [ctypes.c_uint64, vp]
    L.hsmm_status_string.argtypes = [ci]
    L.hsmm_status_string.restype = ctypes.c_char_p
    L.hsmm_last_cuda_error.restype = ci
    L.hsmm_last_error_detail.restype = ctypes.c_char_p
    L.hsmm_version.restype = ci
    L.hsmm_launch_count.argtypes = [ci]
    L.hsmm_launch_count.restype = i64
    for name in EXPORTS:
        if name not in ("hsmm_status_string", "hsmm_last_cuda_error", "hsmm_last_error_detail", "hsmm_version",
                        "hsmm_launch_count"):
            getattr(L, name).restype = ci
    _lib = L
    return L


def status_string(s: int) -> str:
    return lib().hsmm_status_string(int(s)).decode()


def last_cuda_error() -> int:
    return lib().hsmm_last_cuda_error()


def last_error_detail() -> str:
    return lib().hsmm_last_error_detail().decode(errors="replace")


def launch_count(reset: bool = False) -> int:
    return lib().hsmm_launch_count(1 if reset else 0)


def _check(status: int, where: str) -> None:
    if status != SUCCESS:
        raise HsmmError(status, where)


_RAW_STREAM = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream, device: int | None = None) -> int:
    """The CUDA stream handle to launch on: the given stream, else the current stream of
    `device` (read as a raw handle, without building a Stream object per call)."""
    if stream is None:
        if _RAW_STREAM is not None:
            return int(_RAW_STREAM(torch.cuda.current_device() if device is None else device))
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


_N, _T = ord("N"), ord("T")


def _op(t: str) -> int:
    t = t.upper()
    if t not in ("N", "T", "C"):
        raise ValueError(f"op must be 'N', 'T' or 'C', got {t!r}")
    return ord(t)


def colmajor(rows: int, cols: int, dtype=torch.float32, device="cuda", ld: int | None = None):
    """An uninitialised column-major rows x cols tensor (stride(0) == 1, leading dimension ld)."""
    ld = max(1, rows) if ld is None else ld
    base = torch.empty((max(cols, 1), ld), dtype=dtype, device=device)
    return base.t()[:rows, :cols]


def to_colmajor(x: torch.Tensor, ld: int | None = None) -> torch.Tensor:
    out = colmajor(x.shape[0], x.shape[1], x.dtype, x.device, ld)
    out.copy_(x)
    return out


def _ld(x: torch.Tensor) -> int:
    """Leading dimension of a column-major matrix view (element (i, j) at i + j*ld)."""
    if x.dim() != 2:
        raise ValueError("matrices must be 2-D")
    rows, cols = x.shape
    if rows <= 1:
        return max(1, x.stride(1))
    if x.stride(0) != 1:
        raise ValueError("column-major matrix expected (stride(0) == 1)")
    return max(rows, x.stride(1))


_SCALARS: dict = {}


def _scalar_cached(value, dtype_code: int):
    """_scalar for the common alpha / beta values, built once (the library reads them during
    the call; nothing writes to them)."""
    key = (dtype_code, value)
    s = _SCALARS.get(key)
    if s is None:
        s = _scalar(value, dtype_code)
        if len(_SCALARS) < 64:
            _SCALARS[key] = s
    return s


def _scalar(value, dtype_code: int):
    if dtype_code == C_64F:
        z = complex(value)
        return (ctypes.c_double * 2)(z.real, z.imag)
    if dtype_code == R_64F:
        return ctypes.c_double(float(value))
    if dtype_code == R_32I:
        return ctypes.c_int32(int(value))
    return ctypes.c_float(float(value))


def make_config(a: int, b: int, c: int, compute: int = COMPUTE_DEFAULT, slices: int = 0, bits: int = 0,
                workspace: torch.Tensor | None = None, tile_n: int = 0, ring_p: int = 0, ring_k: int = 0) -> Config:
    cfg = Config()
    cfg.a, cfg.b, cfg.c, cfg.compute = a, b, c, compute
    cfg.ozaki_slices, cfg.ozaki_bits, cfg.tile_n = slices, bits, tile_n
    cfg.ring_p, cfg.ring_k = ring_p, ring_k
    if workspace is not None:
        cfg.workspace = workspace.data_ptr()
        cfg.workspace_bytes = workspace.numel() * workspace.element_size()
    return cfg


def workspace_size(cfg: Config, transA="N", transB="N", m=0, n=0, k=0) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().hsmm_workspace_size(ctypes.byref(cfg), _op(transA), _op(transB), m, n, k, ctypes.byref(out)),
           "hsmm_workspace_size")
    return out.value


_CONFIGS: dict = {}
_SCALAR_CODE = {torch.float64: R_64F, torch.complex128: C_64F}


def gemm(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, transA="N", transB="N", alpha=1.0, beta=0.0,
         compute: int = COMPUTE_DEFAULT, slices: int = 0, bits: int = 0, workspace: torch.Tensor | None = None,
         tile_n: int = 0, ring_p: int = 0, ring_k: int = 0, stream=None) -> torch.Tensor:
    """C <- alpha*op(A)*op(B) + beta*C on column-major CUDA tensors (hsmm_gemm).

    ring_p != 0 selects the ring order of Algorithm 2 on clusters of ring_p CTAs with ring_k
    auxiliary accumulators (BF16 in, FP32 out)."""
    m, n = C.shape
    k = A.shape[1] if transA.upper() == "N" else A.shape[0]
    key = (_TORCH2H[A.dtype], _TORCH2H[B.dtype], _TORCH2H[C.dtype], compute, slices, bits, tile_n, ring_p, ring_k)
    if compute == COMPUTE_64F_OZAKI and workspace is None:   # real or complex FP64-accurate form
        cfg = make_config(*key[:6], None, *key[6:])
        need = workspace_size(cfg, transA, transB, m, n, k)
        workspace = torch.empty(need, dtype=torch.uint8, device=C.device)
    if workspace is not None:
        cfg = make_config(*key[:6], workspace, *key[6:])
    else:   # no workspace: a config per key, built once (the library only reads it)
        cfg = _CONFIGS.get(key)
        if cfg is None:
            cfg = _CONFIGS[key] = make_config(*key[:6], None, *key[6:])
    sc = _SCALAR_CODE.get(C.dtype, R_32F)
    al, be = _scalar_cached(alpha, sc), _scalar_cached(beta, sc)
    st = lib().hsmm_gemm(ctypes.byref(cfg), _op(transA), _op(transB), m, n, k, ctypes.byref(al), A.data_ptr(),
                         _ld(A), B.data_ptr(), _ld(B), ctypes.byref(be), C.data_ptr(), _ld(C),
                         _stream(stream, C.device.index))
    _check(st, "hsmm_gemm")
    return C


def gemm_host(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, transA="N", transB="N", alpha=1.0, beta=0.0,
              compute: int = COMPUTE_DEFAULT, slices: int = 0, bits: int = 0, workspace: torch.Tensor | None = None,
              device=None, stream=None) -> torch.Tensor:
    """hsmm_gemm_host: C <- alpha*op(A)*op(B) + beta*C with A, B, C column-major HOST tensors (page-locked
    memory lets the copies overlap the computation); the device workspace holds the device copies."""
    for t in (A, B, C):
        if t.is_cuda:
            raise ValueError("gemm_host takes host tensors")
    m, n = C.shape
    k = A.shape[1] if transA.upper() == "N" else A.shape[0]
    cfg = make_config(_TORCH2H[A.dtype], _TORCH2H[B.dtype], _TORCH2H[C.dtype], compute, slices, bits)
    if workspace is None:
        workspace = torch.empty(gemm_host_workspace_size(cfg, transA, transB, m, n, k), dtype=torch.uint8,
                                device=device or "cuda")
    cfg.workspace = workspace.data_ptr()
    cfg.workspace_bytes = workspace.numel() * workspace.element_size()
    sc = {torch.float64: R_64F, torch.complex128: C_64F}.get(C.dtype, R_32F)
    al, be = _scalar(alpha, sc), _scalar(beta, sc)
    st = lib().hsmm_gemm_host(ctypes.byref(cfg), _op(transA), _op(transB), m, n, k, ctypes.byref(al), A.data_ptr(),
                              _ld(A), B.data_ptr(), _ld(B), ctypes.byref(be), C.data_ptr(), _ld(C), _stream(stream))
    _check(st, "hsmm_gemm_host")
    return C


def gemm_host_workspace_size(cfg: Config, transA="N", transB="N", m=0, n=0, k=0) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().hsmm_gemm_host_workspace_size(ctypes.byref(cfg), _op(transA), _op(transB), m, n, k,
                                               ctypes.byref(out)), "hsmm_gemm_host_workspace_size")
    return out.value


def nbody(x: torch.Tensor, z: torch.Tensor | None = None, eps2: float = 0.0, out: torch.Tensor | None = None,
          ring_p: int = 0, ring_k: int = 0, stream=None) -> torch.Tensor:
    """hsmm_nbody: a_i = sum_j m_j (r_j - r_i) / (|r_j - r_i|^2 + eps2)^(3/2) for float32 CUDA tensors
    x (nx, 4) and z (nz, 4) of (px, py, pz, m); returns (nx, 4) (ax, ay, az, 0).  ring_p != 0: the
    hyper-systolic schedule on clusters of ring_p CTAs with ring_k replicas."""
    z = x if z is None else z
    for t in (x, z):
        if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 4 or not t.is_contiguous():
            raise ValueError("bodies must be contiguous float32 tensors of shape (n, 4)")
    if out is None:
        out = torch.empty_like(x)
    _check(lib().hsmm_nbody(x.shape[0], z.shape[0], x.data_ptr(), z.data_ptr(), float(eps2), out.data_ptr(),
                            int(ring_p), int(ring_k), _stream(stream)), "hsmm_nbody")
    return out


def matmul(a: torch.Tensor, b: torch.Tensor, out: torch.Tensor | None = None, trans_a=False, trans_b=False,
           out_dtype=None, **kw) -> torch.Tensor:
    """Row-major C = op(a) @ op(b) through the column-major library: C^T = op(b)^T op(a)^T.

    a, b, out are contiguous row-major tensors; trans_* select a.T / b.T without copies.
    """
    if not (a.is_contiguous() and b.is_contiguous()):
        raise ValueError("matmul expects contiguous row-major operands")
    m = a.shape[1] if trans_a else a.shape[0]
    n = b.shape[0] if trans_b else b.shape[1]
    if out is None:
        dt = out_dtype or (torch.float32 if a.dtype == torch.bfloat16 else a.dtype)
        out = torch.empty((m, n), dtype=dt, device=a.device)
    if kw or a.dtype != torch.bfloat16 or b.dtype != torch.bfloat16 or not out.is_contiguous() or \
            out.shape != (m, n):
        # the column-major views: row-major X (r x c) is X^T (c x r) with ld = c
        Bv, Av, Cv = b.t(), a.t(), out.t()
        gemm(Bv, Av, Cv, "T" if trans_b else "N", "T" if trans_a else "N", **kw)
        return out
    # the same call without building the three views (this is the per-step path of the
    # autograd Function): C^T (n x m, ld n) = op(b)^T (n x k, ld b.shape[1]) op(a)^T (k x m, ld a.shape[1])
    k = a.shape[0] if trans_a else a.shape[1]
    key = (_TORCH2H[a.dtype], _TORCH2H[b.dtype], _TORCH2H[out.dtype], COMPUTE_DEFAULT, 0, 0, 0, 0, 0)
    cfg = _CONFIGS.get(key)
    if cfg is None:
        cfg = _CONFIGS[key] = make_config(*key[:6], None, *key[6:])
    one, zero = _scalar_cached(1.0, R_32F), _scalar_cached(0.0, R_32F)
    st = lib().hsmm_gemm(ctypes.byref(cfg), _T if trans_b else _N, _T if trans_a else _N, n, m, k, ctypes.byref(one),
                         b.data_ptr(), max(1, b.shape[1]), a.data_ptr(), max(1, a.shape[1]), ctypes.byref(zero),
                         out.data_ptr(), max(1, n), _stream(None, out.device.index))
    _check(st, "hsmm_gemm")
    return out


def gemv_workspace_size(dtype_a: int, trans: str, m: int, n: int) -> int:
    cfg = make_config(dtype_a, dtype_a, R_32F if dtype_a == R_32F else R_32I)
    out = ctypes.c_size_t(0)
    _check(lib().hsmm_gemv_workspace_size(ctypes.byref(cfg), _op(trans), m, n, ctypes.byref(out)),
           "hsmm_gemv_workspace_size")
    return out.value


def gemv(A: torch.Tensor, x: torch.Tensor, y: torch.Tensor, trans="N", alpha=1, beta=0, incx=1, incy=1,
         workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """y <- alpha*op(A)*x + beta*y (hsmm_gemv); A column-major FP32 or INT8, x/y 1-D with strides."""
    m, n = A.shape
    a = _TORCH2H[A.dtype]
    c = _TORCH2H[y.dtype]
    cfg = make_config(a, a, c)
    if workspace is None:
        need = gemv_workspace_size(a, trans, m, n)
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=A.device)
    cfg.workspace = workspace.data_ptr()
    cfg.workspace_bytes = workspace.numel()
    al, be = _scalar(alpha, c), _scalar(beta, c)
    st = lib().hsmm_gemv(ctypes.byref(cfg), _op(trans), m, n, ctypes.byref(al), A.data_ptr(), _ld(A), x.data_ptr(),
                         incx, ctypes.byref(be), y.data_ptr(), incy, _stream(stream))
    _check(st, "hsmm_gemv")
    return y


def gemv_n_noalloc(A: torch.Tensor, x: torch.Tensor, y: torch.Tensor, alpha=1, beta=0, incx=1, incy=1,
                   stream=None) -> torch.Tensor:
    """y <- alpha*A*x + beta*y (op = N) with the library's fixed scratch: no workspace, no allocation.

    For callers that cannot allocate device memory or keep a workspace; calls that
    overlap on the GPU share the scratch and must be serialised (hsmm_gemv_n_noalloc).
    """
    m, n = A.shape
    a = _TORCH2H[A.dtype]
    c = _TORCH2H[y.dtype]
    al, be = _scalar(alpha, c), _scalar(beta, c)
    st = lib().hsmm_gemv_n_noalloc(a, m, n, ctypes.byref(al), A.data_ptr(), _ld(A), x.data_ptr(), incx,
                                   ctypes.byref(be), y.data_ptr(), incy, _stream(stream))
    _check(st, "hsmm_gemv_n_noalloc")
    return y


def ozaki_split(M: torch.Tensor, by_rows: bool, bits: int, slices: int, q: torch.Tensor | None = None,
                expo: torch.Tensor | None = None, stream=None):
    """Splitting step of the FP64-accurate form; returns (expo int32, slices bf16 [s][nv][ldq]).

    q may be a strided view [s][nv][ldq] of planes with a larger pitch (q.stride(0))."""
    rows, cols = M.shape
    nv, length = (rows, cols) if by_rows else (cols, rows)
    ldq = (length + 7) // 8 * 8
    if expo is None:
        expo = torch.empty(nv, dtype=torch.int32, device=M.device)
    if q is None:
        q = torch.empty((slices, nv, ldq), dtype=torch.bfloat16, device=M.device)
    st = lib().hsmm_ozaki_split(rows, cols, M.data_ptr(), _ld(M), 1 if by_rows else 0, bits, slices,
                                expo.data_ptr(), q.data_ptr(), q.stride(1), q.stride(0), _stream(stream))
    _check(st, "hsmm_ozaki_split")
    return expo, q


def ozaki_slice_products(qa: torch.Tensor, qb: torch.Tensor, k: int, bits: int, sd: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """S_d (d = 2..s+1) of split operands qa [s][m][ldq], qb [s][n][ldq] (planes may be strided);
    returns INT32 [s][n][m] (sd may be a strided view of planes of m*n elements)."""
    s, m, ldq = qa.shape
    n = qb.shape[1]
    if sd is None:
        sd = torch.empty((s, n, m), dtype=torch.int32, device=qa.device)
    _check(lib().hsmm_ozaki_slice_products(m, n, k, s, bits, qa.data_ptr(), qa.stride(0), qb.data_ptr(),
                                           qb.stride(0), qa.stride(1), sd.data_ptr(), sd.stride(0),
                                           _stream(stream)), "hsmm_ozaki_slice_products")
    return sd


def ozaki_recombine(sd: torch.Tensor, ea: torch.Tensor, eb: torch.Tensor, C: torch.Tensor, bits: int, alpha=1.0,
                    beta=0.0, stream=None) -> torch.Tensor:
    """C = alpha 2^(ea_i + eb_j) sum_d 2^(-bits d) S_d + beta C from sd [s][n][m] (planes may be strided)."""
    s, n, m = sd.shape
    al, be = ctypes.c_double(alpha), ctypes.c_double(beta)
    _check(lib().hsmm_ozaki_recombine(m, n, s, bits, sd.data_ptr(), sd.stride(0), ea.data_ptr(), eb.data_ptr(),
                                      ctypes.byref(al), ctypes.byref(be), C.data_ptr(), _ld(C), _stream(stream)),
           "hsmm_ozaki_recombine")
    return C


def ring_workspace_size(p: int, K: int, n: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().hsmm_ring_workspace_size(p, K, n, ctypes.byref(out)), "hsmm_ring_workspace_size")
    return out.value


def ring_gemm(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, p: int = 16, K: int = 4,
              workspace: torch.Tensor | None = None, stream=None):
    """C = A*B (n x n FP64, column-major) by the hyper-systolic ring algorithm on p CTAs."""
    n = A.shape[0]
    if workspace is None:
        workspace = torch.empty(max(ring_workspace_size(p, K, n), 16), dtype=torch.uint8, device=A.device)
    st = lib().hsmm_ring_gemm(p, K, n, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(), _ld(C),
                              workspace.data_ptr(), workspace.numel(), _stream(stream))
    _check(st, "hsmm_ring_gemm")
    return C


def _grouped_descs(problems):
    n = len(problems)
    arr = (GemmDesc * max(n, 1))()
    for i, (A, B, C, ta, tb) in enumerate(problems):
        d = arr[i]
        d.transA, d.transB = _op(ta), _op(tb)
        d.m, d.n = C.shape
        d.k = A.shape[1] if ta.upper() == "N" else A.shape[0]
        d.A, d.B, d.C = A.data_ptr(), B.data_ptr(), C.data_ptr()
        d.lda, d.ldb, d.ldc = _ld(A), _ld(B), _ld(C)
    return arr


def gemm_grouped_workspace_size(problems, dtype_ab=R_16BF, dtype_c=R_32F, compute=COMPUTE_DEFAULT, tile_n=0) -> int:
    """Bytes of workspace gemm_grouped needs for these problems (hsmm_gemm_grouped_workspace_size)."""
    cfg = make_config(dtype_ab, dtype_ab, dtype_c, compute, tile_n=tile_n)
    out = ctypes.c_size_t(0)
    _check(lib().hsmm_gemm_grouped_workspace_size(ctypes.byref(cfg), len(problems), _grouped_descs(problems),
                                                  ctypes.byref(out)), "hsmm_gemm_grouped_workspace_size")
    return out.value


def gemm_grouped(problems, dtype_ab=R_16BF, dtype_c=R_32F, compute=COMPUTE_DEFAULT, alpha=1.0, beta=0.0,
                 workspace: torch.Tensor | None = None, tile_n=0, stream=None):
    """One grouped launch of (A, B, C, transA, transB) column-major problems (hsmm_gemm_grouped);
    the descriptors go into `workspace` (allocated here through torch when not given)."""
    if workspace is None:
        need = gemm_grouped_workspace_size(problems, dtype_ab, dtype_c, compute, tile_n)
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=problems[0][2].device)
    cfg = make_config(dtype_ab, dtype_ab, dtype_c, compute, tile_n=tile_n)
    cfg.workspace = workspace.data_ptr()
    cfg.workspace_bytes = workspace.numel()
    al, be = ctypes.c_float(alpha), ctypes.c_float(beta)
    _check(lib().hsmm_gemm_grouped(ctypes.byref(cfg), len(problems), _grouped_descs(problems), ctypes.byref(al),
                                   ctypes.byref(be), _stream(stream)), "hsmm_gemm_grouped")


class GroupedPlan:
    """A grouped launch of independent column-major products (hsmm_grouped_plan_*)."""

    def __init__(self, problems, dtype_ab=R_16BF, dtype_c=R_32F, compute=COMPUTE_DEFAULT, tile_n=0,
                 tile_n_per_problem=None, schedule=1):
        """problems: list of (A, B, C, transA, transB) with column-major CUDA tensors.

        tile_n_per_problem / schedule: the autotuner's choices (see hsmm_grouped_plan_create_ex).
        """
        self.problems = list(problems)          # keep the tensors alive
        n = len(self.problems)
        arr = _grouped_descs(self.problems)
        self._descs = arr
        cfg = make_config(dtype_ab, dtype_ab, dtype_c, compute, tile_n=tile_n)
        h = ctypes.c_void_p(0)
        per = None
        if tile_n_per_problem is not None:
            per = (ctypes.c_int * max(n, 1))(*[int(v) for v in tile_n_per_problem])
        _check(lib().hsmm_grouped_plan_create_ex(ctypes.byref(cfg), n, arr, per, int(schedule), ctypes.byref(h)),
               "hsmm_grouped_plan_create_ex")
        self.handle = h
        self.count = n

    def launch(self, alpha=1.0, beta=0.0, stream=None):
        al, be = ctypes.c_float(alpha), ctypes.c_float(beta)
        _check(lib().hsmm_grouped_plan_launch(self.handle, ctypes.byref(al), ctypes.byref(be), _stream(stream)),
               "hsmm_grouped_plan_launch")

    def info(self):
        tiles = ctypes.c_int64(0)
        per = (ctypes.c_int * max(self.count, 1))()
        _check(lib().hsmm_grouped_plan_info(self.handle, ctypes.byref(tiles), per), "hsmm_grouped_plan_info")
        return tiles.value, list(per)[: self.count]

    def close(self):
        if getattr(self, "handle", None):
            lib().hsmm_grouped_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sync_status(stream=None) -> int:
    return lib().hsmm_sync_status(_stream(stream))


def set_wait_timeout_ns(ns: int) -> None:
    _check(lib().hsmm_set_wait_timeout_ns(int(ns)), "hsmm_set_wait_timeout_ns")


def selftest_timeout(timeout_ns: int, stream=None) -> int:
    return lib().hsmm_selftest_timeout(int(timeout_ns), _stream(stream))
