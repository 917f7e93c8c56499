"""Oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU implementations (FP64, exact integers) of
what the hsmm hot path computes, written from the paper "Hyper-Systolic Matrix
Multiplication" (Lippert, Petkov, Palazzari, Schilling) and, for the precision
form, from the published error-free splitting of Ozaki, Ogita, Oishi and Rump.

Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path and never imports it.

All matrices are NumPy arrays in column-major (Fortran) order; ``op`` flags are
'N' or 'T' as in BLAS ('C', the conjugate transpose, for complex matrices).  The C source is ``oracle.c`` beside this file; the
function-level parity status (pinned / unpinned) is listed in its header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

_i64 = ctypes.c_int64
_f64 = ctypes.c_double
_vp = ctypes.c_void_p
_ch = ctypes.c_char
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.ora_threads.restype = _int
            L.ora_set_threads.argtypes = [_int]
            L.ora_gemm_f64.argtypes = [_ch, _ch, _i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64, _vp, _i64]
            L.ora_gemm_i64.argtypes = [_ch, _ch, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64]
            L.ora_zgemm.argtypes = [_ch, _ch, _i64, _i64, _i64, _vp, _vp, _i64, _vp, _i64, _vp, _vp, _i64]
            L.ora_nbody_direct.argtypes = [_int, _i64, _i64, _vp, _vp, _f64, _vp]
            L.ora_nbody_hsys.argtypes = [_int, _int, _int, _int, _i64, _vp, _vp, _f64, _vp, _vp, _vp]
            L.ora_nbody_hsys.restype = _int
            L.ora_gemm_rows_f64.argtypes = [_ch, _ch, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _i64, _vp, _vp]
            L.ora_dot2_rows.argtypes = [_ch, _ch, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _i64, _vp, _vp]
            L.ora_dot2.argtypes = [_vp, _vp, _i64]
            L.ora_dot2.restype = _f64
            L.ora_gemv_f64.argtypes = [_ch, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64, _vp, _i64]
            L.ora_gemv_i8.argtypes = [_ch, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _i64, _vp, _i64, _vp]
            L.ora_ring_systolic.argtypes = [_int, _int, _vp, _vp, _vp, _vp, _vp]
            L.ora_ring_systolic.restype = _int
            L.ora_ring_hsmm.argtypes = [_int, _int, _int, _vp, _vp, _vp, _vp, _vp, _int]
            L.ora_ring_hsmm.restype = _int
            L.ora_regular_base.argtypes = [_int, _int, _vp, _vp, _vp, _vp, _vp]
            L.ora_regular_base.restype = _int
            L.ora_skew_row.argtypes = [_int, _int, _int]
            L.ora_skew_row.restype = _int
            L.ora_preshift_stride.argtypes = [_int, _int, _int]
            L.ora_preshift_stride.restype = _int
            L.ora_ozaki_split.argtypes = [_i64, _i64, _vp, _i64, _int, _int, _int, _vp, _vp]
            L.ora_ozaki_diagonals.argtypes = [_i64, _i64, _i64, _int, _vp, _vp, _vp]
            L.ora_ozaki_gemm.argtypes = [_ch, _ch, _i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64, _vp,
                                         _i64, _int, _int]
            _lib = L
    return _lib


def threads() -> int:
    return lib().ora_threads()


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def _f(a, dtype=np.float64):
    a = np.asarray(a, dtype=dtype)
    return np.asfortranarray(a) if a.ndim == 2 else np.ascontiguousarray(a)


def _p(a):
    return a.ctypes.data_as(_vp)


def _b(t: str) -> bytes:
    return t.encode()


def _opshape(M, t):
    return M.shape if t in "Nn" else (M.shape[1], M.shape[0])


def gemm(A, B, ta="N", tb="N", alpha=1.0, beta=0.0, C=None):
    """C <- alpha*op(A)*op(B) + beta*C in FP64, Eq. PRODUCT with sequential k."""
    A = _f(A); B = _f(B)
    m, k = _opshape(A, ta)
    k2, n = _opshape(B, tb)
    assert k == k2, (A.shape, B.shape, ta, tb)
    out = _f(C) .copy(order="F") if C is not None else np.zeros((m, n), order="F")
    lib().ora_gemm_f64(_b(ta), _b(tb), m, n, k, float(alpha), _p(A), max(1, A.shape[0]), _p(B),
                       max(1, B.shape[0]), float(beta), _p(out), max(1, m))
    return out


def gemm_i64(A, B, ta="N", tb="N"):
    """Exact integer product op(A)*op(B)."""
    A = _f(A, np.int64); B = _f(B, np.int64)
    m, k = _opshape(A, ta)
    k2, n = _opshape(B, tb)
    assert k == k2
    out = np.zeros((m, n), dtype=np.int64, order="F")
    lib().ora_gemm_i64(_b(ta), _b(tb), m, n, k, _p(A), max(1, A.shape[0]), _p(B), max(1, B.shape[0]),
                       _p(out), max(1, m))
    return out


def _zopshape(M, t):
    return M.shape if t in "Nn" else (M.shape[1], M.shape[0])


def zgemm(A, B, ta="N", tb="N", alpha=1.0, beta=0.0, C=None):
    """C <- alpha*op(A)*op(B) + beta*C for complex128 matrices, op in N/T/C, sequential k."""
    A = _f(A, np.complex128); B = _f(B, np.complex128)
    m, k = _zopshape(A, ta)
    k2, n = _zopshape(B, tb)
    assert k == k2, (A.shape, B.shape, ta, tb)
    out = _f(C, np.complex128).copy(order="F") if C is not None else np.zeros((m, n), np.complex128, order="F")
    al = np.array([complex(alpha).real, complex(alpha).imag])
    be = np.array([complex(beta).real, complex(beta).imag])
    lib().ora_zgemm(_b(ta), _b(tb), m, n, k, _p(al), _p(A), max(1, A.shape[0]), _p(B), max(1, B.shape[0]),
                    _p(be), _p(out), max(1, m))
    return out


def zop(M, t):
    """op(M) of a complex matrix as an explicit array (N, T or C)."""
    M = np.asarray(M, np.complex128)
    return M if t in "Nn" else (M.T if t in "Tt" else M.conj().T)


def zembed(A, B, ta="N", tb="N"):
    """The real form of the complex product op(A) op(B):
        A' = [Re op(A), Im op(A)]                      (m x 2k)
        B'' = [[Re op(B), Im op(B)], [-Im op(B), Re op(B)]]   (2k x 2n)
    so that A' B'' = [Re(op(A) op(B)), Im(op(A) op(B))]: column j of the first half is
    sum_k Re a Re b - Im a Im b, of the second half sum_k Re a Im b + Im a Re b, the
    definition of the complex product with the two real sums of each part joined."""
    a, b = zop(A, ta), zop(B, tb)
    Ap = np.asfortranarray(np.hstack([a.real, a.imag]))
    Bpp = np.asfortranarray(np.block([[b.real, b.imag], [-b.imag, b.real]]))
    return Ap, Bpp


def zgemm_rows(A, B, rows, ta="N", tb="N", accurate=True):
    """Selected rows of op(A) op(B) (complex) from the real form: Dot2 sums of length 2k."""
    Ap, Bpp = zembed(A, B, ta, tb)
    r = gemm_rows(Ap, Bpp, rows, accurate=accurate)
    n = Bpp.shape[1] // 2
    return r[:, :n] + 1j * r[:, n:]


def gemm_rows(A, B, rows, ta="N", tb="N", accurate=False):
    """Selected rows of op(A)*op(B): plain sequential sums, or Dot2 when accurate."""
    A = _f(A); B = _f(B)
    m, k = _opshape(A, ta)
    k2, n = _opshape(B, tb)
    assert k == k2
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((len(rows), n), dtype=np.float64)
    fn = lib().ora_dot2_rows if accurate else lib().ora_gemm_rows_f64
    fn(_b(ta), _b(tb), m, n, k, _p(A), max(1, A.shape[0]), _p(B), max(1, B.shape[0]), len(rows), _p(rows),
       _p(out))
    return out


def dot2(x, y):
    x = _f(x); y = _f(y)
    return lib().ora_dot2(_p(x), _p(y), len(x))


def gemv(A, x, trans="N", alpha=1.0, beta=0.0, y=None, incx=1, incy=1):
    """y <- alpha*op(A)*x + beta*y in FP64 (x and y given with their strides)."""
    A = _f(A); x = _f(x)
    m, n = A.shape
    leny = m if trans in "Nn" else n
    yy = _f(y).copy() if y is not None else np.zeros(leny * incy)
    lib().ora_gemv_f64(_b(trans), m, n, float(alpha), _p(A), max(1, m), _p(x), incx, float(beta), _p(yy), incy)
    return yy


def gemv_i8(A, x, trans="N", alpha=1, beta=0, y=None, incx=1, incy=1):
    """Exact integer y = alpha*op(A)*x + beta*y for INT8 A, x and INT32 y (int64 result)."""
    A = _f(A, np.int8); x = _f(x, np.int8)
    m, n = A.shape
    leny = m if trans in "Nn" else n
    yin = _f(y, np.int32) if y is not None else np.zeros(leny * incy, dtype=np.int32)
    out = np.zeros(leny, dtype=np.int64)
    lib().ora_gemv_i8(_b(trans), m, n, int(alpha), _p(A), max(1, m), _p(x), incx, int(beta), _p(yin), incy,
                      _p(out))
    return out


STAT_KEYS = ("b_rows_shifted", "a_shifts", "c_shifts", "blocks_moved", "pairing_errors", "a_final_ok",
             "b_preshift_events", "shift_events")


def ring_systolic(A, B, p, with_counts=False):
    """Algorithm 1 over p virtual processors on p x p blocks of an n x n product."""
    A = _f(A); B = _f(B)
    n = A.shape[0]
    assert A.shape == (n, n) and B.shape == (n, n) and n % p == 0
    C = np.zeros((n, n), order="F")
    st = np.zeros(8, dtype=np.int64)
    cnt = np.zeros(p * p * p, dtype=np.int32) if with_counts else None
    rc = lib().ora_ring_systolic(p, n // p, _p(A), _p(B), _p(C), _p(st), _p(cnt) if cnt is not None else None)
    assert rc == 0
    stats = dict(zip(STAT_KEYS, (int(v) for v in st)))
    return (C, stats, cnt.reshape(p, p, p)) if with_counts else (C, stats)


def ring_hsmm(A, B, p, K, with_counts=False, planted_nonneg_mod=False):
    """Algorithm 2 (hyper-systolic) over p virtual processors, K*Kt = p."""
    A = _f(A); B = _f(B)
    n = A.shape[0]
    assert A.shape == (n, n) and B.shape == (n, n) and n % p == 0
    C = np.zeros((n, n), order="F")
    st = np.zeros(8, dtype=np.int64)
    cnt = np.zeros(p * p * p, dtype=np.int32) if with_counts else None
    rc = lib().ora_ring_hsmm(p, K, n // p, _p(A), _p(B), _p(C), _p(st), _p(cnt) if cnt is not None else None,
                             1 if planted_nonneg_mod else 0)
    if rc != 0:
        raise ValueError(f"ring_hsmm: invalid p={p}, K={K}")
    stats = dict(zip(STAT_KEYS, (int(v) for v in st)))
    return (C, stats, cnt.reshape(p, p, p)) if with_counts else (C, stats)


def skew_row(p, i, l):
    """Block row held by processor i in slot l (0-based) in skew order."""
    return lib().ora_skew_row(p, i, l)


def preshift_stride(j, K, planted=False):
    """Stride MOD(1-j, K) of the pre-shift of B row j (1-based), Algorithm 2."""
    return lib().ora_preshift_stride(j, K, 1 if planted else 0)


def regular_base(p, K):
    """Regular bases: Section 5.2.1 three-base form and Definition REGULARBASE2."""
    Kt = p // K
    a = np.zeros(Kt, dtype=np.int32); b = np.zeros(K, dtype=np.int32); c = np.zeros(K, dtype=np.int32)
    a2 = np.zeros(K, dtype=np.int32); b2 = np.zeros(Kt, dtype=np.int32)
    rc = lib().ora_regular_base(p, K, _p(a), _p(b), _p(c), _p(a2), _p(b2))
    if rc != 0:
        raise ValueError(f"regular_base: invalid p={p}, K={K}")
    return {"A": a.tolist(), "B": b.tolist(), "C": c.tolist(), "A2": a2.tolist(), "B2": b2.tolist()}


def nbody_direct(x, z, eps2, kind=0):
    """F_i = sum_j f(x_i, z_j) in FP64, j in order; x, z arrays (n, 4) of (px, py, pz, m)."""
    x = np.ascontiguousarray(x, dtype=np.float64); z = np.ascontiguousarray(z, dtype=np.float64)
    F = np.zeros((x.shape[0], 3))
    lib().ora_nbody_direct(int(kind), x.shape[0], z.shape[0], _p(x), _p(z), float(eps2), _p(F))
    return F


def nbody_hsys(x, z, p, K, eps2, kind=0, zstride=0):
    """The hyper-systolic two-array recipe with regular bases on p cells: (F, block-pair counts
    [x block][z block], (replica, z, back) shift counts)."""
    x = np.ascontiguousarray(x, dtype=np.float64); z = np.ascontiguousarray(z, dtype=np.float64)
    n = x.shape[0]
    assert z.shape[0] == n
    F = np.zeros((n, 3))
    cnt = np.zeros((p, p), dtype=np.int32)
    sh = np.zeros(3, dtype=np.int32)
    rc = lib().ora_nbody_hsys(int(kind), int(p), int(K), int(zstride), n, _p(x), _p(z), float(eps2), _p(F),
                              _p(cnt), _p(sh))
    if rc != 0:
        raise ValueError(f"nbody_hsys: invalid p={p}, K={K}, n={n}")
    return F, cnt, tuple(int(v) for v in sh)


def ozaki_split(M, by_rows, beta_bits, s):
    """Error-free splitting into s integer slices (values as float64) and exponents."""
    M = _f(M)
    r, c = M.shape
    nvec = r if by_rows else c
    expo = np.zeros(nvec, dtype=np.int32)
    sl = np.zeros((s, r, c), dtype=np.float64)
    out = np.zeros(s * r * c, dtype=np.float64)
    lib().ora_ozaki_split(r, c, _p(M), max(1, r), 1 if by_rows else 0, beta_bits, s, _p(expo), _p(out))
    for t in range(s):
        sl[t] = out[t * r * c:(t + 1) * r * c].reshape((r, c), order="F")
    return expo, sl


def ozaki_diagonals(A, B, ta="N", tb="N", beta_bits=7, s=7):
    """Exact S_d = sum_{t+u=d} QA_t QB_u (d = 2..s+1) of the split op(A), op(B): int64 [s][m][n]."""
    A = _f(A); B = _f(B)
    Ao = A if ta in "Nn" else np.asfortranarray(A.T)
    Bo = B if tb in "Nn" else np.asfortranarray(B.T)
    m, k = Ao.shape
    n = Bo.shape[1]
    ea, qa = ozaki_split(Ao, True, beta_bits, s)
    eb, qb = ozaki_split(Bo, False, beta_bits, s)
    qa_f = np.ascontiguousarray(np.stack([np.asfortranarray(q).ravel(order="F") for q in qa]))
    qb_f = np.ascontiguousarray(np.stack([np.asfortranarray(q).ravel(order="F") for q in qb]))
    sd = np.zeros(s * m * n, dtype=np.int64)
    lib().ora_ozaki_diagonals(m, n, k, s, _p(qa_f), _p(qb_f), _p(sd))
    out = np.stack([sd[d * m * n:(d + 1) * m * n].reshape((m, n), order="F") for d in range(s)])
    return ea, eb, out


def ozaki_gemm(A, B, ta="N", tb="N", alpha=1.0, beta=0.0, C=None, beta_bits=7, s=7):
    """FP64-accurate product by error-free splitting (exact slice products)."""
    A = _f(A); B = _f(B)
    m, k = _opshape(A, ta)
    k2, n = _opshape(B, tb)
    assert k == k2
    out = _f(C).copy(order="F") if C is not None else np.zeros((m, n), order="F")
    lib().ora_ozaki_gemm(_b(ta), _b(tb), m, n, k, float(alpha), _p(A), max(1, A.shape[0]), _p(B),
                         max(1, B.shape[0]), float(beta), _p(out), max(1, m), int(beta_bits), int(s))
    return out
