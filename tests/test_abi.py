"""The C-ABI library loads and exports every symbol include/hsmm.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hsmm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(hsmm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_cs_9809105_gb300 import build
    return build.build()


def test_header_declares_boundary():
    names = declared_functions()
    for required in ("hsmm_gemm", "hsmm_gemv", "hsmm_gemm_grouped"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_exports(libpath):
    from paper_cs_9809105_gb300 import hsmm
    assert sorted(hsmm.EXPORTS) == sorted(set(hsmm.EXPORTS))
    assert set(hsmm.EXPORTS) <= set(declared_functions())


def test_status_strings_host_only(libpath):
    lib = ctypes.CDLL(libpath)
    lib.hsmm_status_string.restype = ctypes.c_char_p
    assert lib.hsmm_status_string(0) == b"HSMM_STATUS_SUCCESS"
    assert lib.hsmm_status_string(5) == b"HSMM_STATUS_TIMEOUT"
    assert lib.hsmm_status_string(99) == b"HSMM_STATUS_UNKNOWN"


def test_argument_errors_detected_on_host(libpath):
    # invalid arguments are rejected before any CUDA call, so this runs without a GPU
    from paper_cs_9809105_gb300 import hsmm
    L = hsmm.lib()
    cfg = hsmm.make_config(hsmm.R_64F, hsmm.R_64F, hsmm.R_64F)
    one = ctypes.c_double(1.0)
    args = lambda m, n, k, lda, ldb, ldc, ta=ord("N"), tb=ord("N"): (
        ctypes.byref(cfg), ta, tb, m, n, k, ctypes.byref(one), 16, lda, 16, ldb, ctypes.byref(one), 16, ldc, None)
    assert L.hsmm_gemm(*args(-1, 2, 2, 2, 2, 2)) == hsmm.INVALID_VALUE
    assert L.hsmm_gemm(*args(4, 2, 2, 3, 2, 4)) == hsmm.INVALID_VALUE       # lda < m
    assert L.hsmm_gemm(*args(4, 2, 3, 2, 3, 4, ord("T"))) == hsmm.INVALID_VALUE   # lda < k for op T
    assert L.hsmm_gemm(*args(4, 2, 2, 4, 2, 3)) == hsmm.INVALID_VALUE       # ldc < m
    assert L.hsmm_gemm(*args(4, 2, 2, 4, 2, 4, ord("X"))) == hsmm.INVALID_VALUE
    assert L.hsmm_gemm(*args(0, 5, 5, 1, 5, 1)) == hsmm.SUCCESS             # m == 0: nothing to do
    bad = hsmm.make_config(hsmm.R_8I, hsmm.R_8I, hsmm.R_32I)
    assert L.hsmm_gemm(ctypes.byref(bad), ord("N"), ord("N"), 4, 4, 4, ctypes.byref(one), 16, 4, 16, 4,
                       ctypes.byref(one), 16, 4, None) == hsmm.NOT_SUPPORTED
    g = hsmm.make_config(hsmm.R_32F, hsmm.R_32F, hsmm.R_32F)
    onef = ctypes.c_float(1.0)
    assert L.hsmm_gemv(ctypes.byref(g), ord("N"), 4, 4, ctypes.byref(onef), 16, 4, 16, 0, ctypes.byref(onef), 16, 1,
                       None) == hsmm.INVALID_VALUE                           # incx == 0
    assert L.hsmm_gemv(ctypes.byref(g), ord("N"), 4, 4, ctypes.byref(onef), 16, 4, 16, -1, ctypes.byref(onef), 16, 1,
                       None) == hsmm.NOT_SUPPORTED
    # ring order of the tensor-core product: cluster size and accumulator count checked on the host
    b16 = lambda p, k: hsmm.make_config(hsmm.R_16BF, hsmm.R_16BF, hsmm.R_32F, ring_p=p, ring_k=k)
    ring = lambda c: L.hsmm_gemm(ctypes.byref(c), ord("N"), ord("N"), 256, 256, 256, ctypes.byref(onef), 16, 256, 16,
                                 256, ctypes.byref(onef), 16, 256, None)
    for p, k in ((3, 1), (4, 3), (2, 4), (32, 0), (8, 8), (-1, 0), (4, -1)):
        assert ring(b16(p, k)) == hsmm.INVALID_VALUE, (p, k)
    assert ring(hsmm.make_config(hsmm.R_16BF, hsmm.R_16BF, hsmm.R_16BF, ring_p=4)) == hsmm.NOT_SUPPORTED
    r = b16(4, 2)
    r.reserved[0] = 1
    assert ring(r) == hsmm.INVALID_VALUE
    # two-array n^2 problem: schedule and argument checks on the host
    nb = lambda nx, nz, x, eps2, p, k: L.hsmm_nbody(nx, nz, x, x, ctypes.c_float(eps2), 16, p, k, None)
    assert nb(10, 10, 16, -1.0, 0, 0) == hsmm.INVALID_VALUE
    for p, k in ((3, 0), (4, 3), (2, 4), (32, 0), (8, 8)):
        assert nb(10, 10, 16, 0.0, p, k) == hsmm.INVALID_VALUE, (p, k)
    assert nb(10, 10, 8, 0.0, 0, 0) == hsmm.NOT_SUPPORTED                      # not 16-byte aligned
    assert nb(0, 10, 16, 0.0, 4, 2) == hsmm.SUCCESS                            # nothing to do
    assert L.hsmm_ring_gemm(16, 3, 512, 16, 512, 16, 512, 16, 512, 16, 0, None) == hsmm.INVALID_VALUE  # K does not divide p
    assert L.hsmm_ring_gemm(16, 4, 1024, 16, 1024, 16, 1024, 16, 1024, 16, 0, None) == hsmm.NOT_SUPPORTED  # b = 64
    # grouped plans: the schedule is 0 or 1
    gb = hsmm.make_config(hsmm.R_16BF, hsmm.R_16BF, hsmm.R_32F)
    plan = ctypes.c_void_p()
    for sched in (-1, 2):
        assert L.hsmm_grouped_plan_create_ex(ctypes.byref(gb), 0, None, None, sched, ctypes.byref(plan)) == \
            hsmm.INVALID_VALUE, sched
    # tile widths: 0 (automatic) or a multiple of 32 up to 256, checked before any device work
    desc = (hsmm.GemmDesc * 1)()
    d = desc[0]
    d.transA, d.transB, d.m, d.n, d.k = ord("N"), ord("N"), 4, 4, 4
    d.A, d.B, d.C, d.lda, d.ldb, d.ldc = 16, 16, 16, 8, 8, 8
    for w in (-32, 100, 288, 16):
        width = (ctypes.c_int * 1)(w)
        assert L.hsmm_grouped_plan_create_ex(ctypes.byref(gb), 1, desc, width, 1, ctypes.byref(plan)) == \
            hsmm.INVALID_VALUE, w


def declared_param_counts():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(hsmm_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_header(libpath):
    from paper_cs_9809105_gb300 import hsmm
    L = hsmm.lib()
    counts = declared_param_counts()
    for name in hsmm.EXPORTS:
        at = getattr(L, name).argtypes
        expected = counts[name]
        got = 0 if at is None else len(at)
        assert got == expected, (name, got, expected)


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of hsmm_config_t and hsmm_gemm_desc_t have the C compiler's offsets and sizes."""
    import shutil
    import subprocess
    from paper_cs_9809105_gb300 import hsmm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"hsmm_config_t": hsmm.Config, "hsmm_gemm_desc_t": hsmm.GemmDesc}
    lines = ['#include <stdio.h>', '#include "hsmm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def test_host_product_workspace_sizes(libpath):
    """hsmm_gemm_host's workspace (computed on the host): device copies of A, B and C with
    leading dimensions padded to 16 elements, plus, for the FP64-accurate form, the slices of
    all of op(A) but of one column panel of op(B), and the sums of one column panel of C."""
    from paper_cs_9809105_gb300 import hsmm
    f64 = hsmm.make_config(hsmm.R_64F, hsmm.R_64F, hsmm.R_64F, hsmm.COMPUTE_64F_NATIVE)
    up = lambda v: (v + 255) // 256 * 256
    pad = lambda r: (max(r, 1) + 15) // 16 * 16
    for m, n, k in ((8192, 8192, 8192), (100, 37, 5), (4300, 4200, 40)):
        assert hsmm.gemm_host_workspace_size(f64, "N", "N", m, n, k) == \
            up(pad(m) * k * 8) + up(pad(k) * n * 8) + up(pad(m) * n * 8)
    assert hsmm.gemm_host_workspace_size(f64, "T", "T", 100, 37, 5) == \
        up(pad(5) * 100 * 8) + up(pad(37) * 5 * 8) + up(pad(100) * 37 * 8)
    acc = hsmm.make_config(hsmm.R_64F, hsmm.R_64F, hsmm.R_64F, hsmm.COMPUTE_64F_OZAKI, 7, 7)
    m = n = k = 8192
    copies = 3 * m * n * 8
    host = hsmm.gemm_host_workspace_size(acc, "N", "N", m, n, k)
    whole = hsmm.workspace_size(acc, "N", "N", m, n, k)
    half = hsmm.workspace_size(acc, "N", "N", m, n // 2, k)     # one of the two column panels
    assert host - copies == half
    assert half < whole
