"""GPU parity of the grouped persistent launch (many uneven products, one launch, CUDA graph)."""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import dev_bf16_colmajor, dev_colmajor, hsmm, padded, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.fixture(params=["pair", "single"])
def grouped_kernel(request, monkeypatch):
    """The grouped kernels: 256-row tiles on CTA pairs (default) and 128-row tiles on one CTA."""
    monkeypatch.setenv("HSMM_GROUPED_KERNEL", request.param)
    return request.param


def make_problems(shapes, seed, trans=("N", "N"), dtype="bf16", c_aligned=False, out=torch.float32):
    """c_aligned: ldc a multiple of 16 bytes, so C leaves the kernel by TMA stores of 32 x 32
    blocks; otherwise ldc = m + 1 and the element-wise epilogue writes it."""
    probs, host = [], []
    h = hsmm()
    ta, tb = trans
    for q, (m, n, k) in enumerate(shapes):
        sa = (m, k) if ta == "N" else (k, m)
        sb = (k, n) if tb == "N" else (n, k)
        if dtype == "bf16":
            Ab, Bb = W.uniform_bf16(sa, seed + 2 * q), W.uniform_bf16(sb, seed + 2 * q + 1)
            A64, B64 = W.bf16_bits_to_f64(Ab), W.bf16_bits_to_f64(Bb)
            dA = dev_bf16_colmajor(Ab, ld=padded(sa[0]))
            dB = dev_bf16_colmajor(Bb, ld=padded(sb[0]))
        else:
            A32, B32 = W.uniform_f32(sa, seed + 2 * q), W.uniform_f32(sb, seed + 2 * q + 1)
            A64, B64 = A32.astype(np.float64), B32.astype(np.float64)
            dA = dev_colmajor(A32, ld=padded(sa[0], 4))
            dB = dev_colmajor(B32, ld=padded(sb[0], 4))
        ldc = padded(m, 8) + 8 if c_aligned else m + 1
        # NaN everywhere in C's storage, the padding rows beyond m included: check() requires
        # that the padding is still NaN afterwards
        dC = torch.full((n, ldc), float("nan"), dtype=out, device="cuda")[:, :m].t()
        probs.append((dA, dB, dC, ta, tb))
        host.append((A64, B64))
    return probs, host


def check(ora, probs, host, ta, tb, tol_fn):
    for (dA, dB, dC, _, _), (A64, B64) in zip(probs, host):
        if dC._base is not None:   # nothing written into the padding rows of C
            assert torch.isnan(dC._base[:, dC.shape[0]:].float()).all(), "padding rows beyond m were written"
        got = dC.double().cpu().numpy()
        want = ora.gemm(A64, B64, ta, tb)
        mag = ora.gemm(np.abs(A64), np.abs(B64), ta, tb)
        k = A64.shape[1] if ta == "N" else A64.shape[0]
        assert (np.abs(got - want) <= tol_fn(k) * mag).all()


SHAPES = [(64, 64, 64), (300, 200, 100), (129, 257, 65), (1000, 70, 900), (64, 2048, 64), (513, 512, 1024),
          (77, 130, 333), (256, 256, 8)]


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("c_aligned", [False, True])
def test_grouped_bf16(ora, ta, tb, schedule, c_aligned, grouped_kernel):
    h = hsmm()
    probs, host = make_problems(SHAPES, 500, (ta, tb), c_aligned=c_aligned)
    plan = h.GroupedPlan(probs, schedule=schedule)
    plan.launch()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    check(ora, probs, host, ta, tb, lambda k: 2 * k * 2.0 ** -24)
    tiles, per = plan.info()
    assert tiles > 0
    if grouped_kernel == "pair" and tb == "N":   # K-major B on CTA pairs: multiples of 32 columns
        assert all(w % 32 == 0 and 32 <= w <= 256 for w in per), per
    else:
        assert set(per) <= {128, 256}
    plan.close()


@pytest.mark.parametrize("widths", [[32, 64, 96, 160, 192, 224, 256, 128], [96] * 8])
def test_grouped_explicit_widths(ora, widths):
    """Tile widths of any multiple of 32 on CTA pairs with K-major B (ragged n, m and k included)."""
    h = hsmm()
    probs, host = make_problems(SHAPES, 650, c_aligned=True)
    plan = h.GroupedPlan(probs, tile_n_per_problem=widths, schedule=1)
    plan.launch()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    check(ora, probs, host, "N", "N", lambda k: 2 * k * 2.0 ** -24)
    assert plan.info()[1] == widths
    plan.close()


def test_grouped_widths_refused_where_not_supported(monkeypatch):
    """96-column tiles need CTA pairs and a K-major B: MN-major B or the one-CTA kernel refuse them."""
    h = hsmm()
    probs, _ = make_problems(SHAPES[:2], 660, ("N", "T"))
    with pytest.raises(h.HsmmError):
        h.GroupedPlan(probs, tile_n_per_problem=[96, 96])
    monkeypatch.setenv("HSMM_GROUPED_KERNEL", "single")
    probs, _ = make_problems(SHAPES[:2], 661)
    with pytest.raises(h.HsmmError):
        h.GroupedPlan(probs, tile_n_per_problem=[96, 96])


def test_grouped_tile_widths_and_beta(ora, grouped_kernel):
    h = hsmm()
    probs, host = make_problems(SHAPES, 600)
    for _, _, dC, _, _ in probs:
        dC.fill_(1.0)
    plan = h.GroupedPlan(probs, tile_n_per_problem=[128, 256] * (len(SHAPES) // 2), schedule=0)
    plan.launch(alpha=2.0, beta=-1.0)
    torch.cuda.synchronize()
    for (dA, dB, dC, _, _), (A64, B64) in zip(probs, host):
        want = 2.0 * ora.gemm(A64, B64) - 1.0
        mag = 2.0 * ora.gemm(np.abs(A64), np.abs(B64)) + 1.0
        k = A64.shape[1]
        assert (np.abs(dC.double().cpu().numpy() - want) <= 2 * k * 2.0 ** -24 * mag).all()
    assert plan.info()[1] == [128, 256] * (len(SHAPES) // 2)


@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("c_aligned", [False, True])
def test_grouped_tf32(ora, ta, tb, c_aligned, grouped_kernel):
    """The FP32/TF32 variant of the batching form, every operand form (NN is the workload's)."""
    h = hsmm()
    probs, host = make_problems(SHAPES, 700, (ta, tb), dtype="f32", c_aligned=c_aligned)
    plan = h.GroupedPlan(probs, h.R_32F, h.R_32F, h.COMPUTE_32F_FAST_TF32)
    plan.launch()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    check(ora, probs, host, ta, tb, lambda k: 2.0 ** -9 + k * 2.0 ** -23)
    plan.close()


def test_grouped_graph_autotune_workload_sample(ora, tmp_path):
    """The 512-problem workload (log-uniform shapes): tuned plan captured in a CUDA graph;
    every problem checked on sampled rows."""
    from paper_cs_9809105_gb300.grouped import GroupedGemm
    h = hsmm()
    shapes = W.grouped_shapes()
    probs, host = make_problems([tuple(int(v) for v in s) for s in shapes], 800, c_aligned=True)
    gg = GroupedGemm(probs, tune=True, table_path=str(tmp_path / "tune.json"))
    gg.replay()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    g = W.rng(9)
    for (dA, dB, dC, _, _), (A64, B64) in zip(probs, host):
        m = A64.shape[0]
        rows = g.choice(m, size=min(4, m), replace=False)
        want = ora.gemm_rows(A64, B64, rows)
        mag = ora.gemm_rows(np.abs(A64), np.abs(B64), rows)
        got = dC[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        k = A64.shape[1]
        assert (np.abs(got - want) <= 2 * k * 2.0 ** -24 * mag).all()


@pytest.mark.parametrize("c_aligned", [False, True])
def test_grouped_bf16_output(ora, c_aligned, grouped_kernel):
    """BF16 C: one rounding of the FP32 accumulator, through either epilogue path."""
    h = hsmm()
    probs, host = make_problems(SHAPES, 900, c_aligned=c_aligned, out=torch.bfloat16)
    plan = h.GroupedPlan(probs, h.R_16BF, h.R_16BF)
    plan.launch(alpha=0.5)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    for (dA, dB, dC, _, _), (A64, B64) in zip(probs, host):
        want = 0.5 * ora.gemm(A64, B64)
        mag = 0.5 * ora.gemm(np.abs(A64), np.abs(B64))
        k = A64.shape[1]
        got = dC.double().cpu().numpy()
        assert (np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 2 * k * 2.0 ** -24 * mag).all()
    plan.close()


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_gemm_grouped_workspace_call(ora, dtype):
    """hsmm_gemm_grouped without a plan: the descriptors go into the caller's workspace (nothing
    allocated), every operand form in one launch, against the oracle."""
    h = hsmm()
    shapes = SHAPES
    forms = [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")]
    probs, hosts, tr = [], [], []
    for q, sh in enumerate(shapes):
        ta, tb = forms[q % 4]
        p, hh = make_problems([sh], 1000 + 7 * q, (ta, tb), dtype=dtype, c_aligned=(q % 2 == 0))
        probs += p
        hosts += hh
        tr.append((ta, tb))
    ab = h.R_16BF if dtype == "bf16" else h.R_32F
    comp = h.COMPUTE_DEFAULT if dtype == "bf16" else h.COMPUTE_32F_FAST_TF32
    need = h.gemm_grouped_workspace_size(probs, ab, h.R_32F, comp)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h.gemm_grouped(probs, ab, h.R_32F, comp, workspace=ws)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    tol = (lambda k: 2 * k * 2.0 ** -24) if dtype == "bf16" else (lambda k: 2.0 ** -9 + k * 2.0 ** -23)
    for prob, hh, (ta, tb) in zip(probs, hosts, tr):
        check(ora, [prob], [hh], ta, tb, tol)
    # 64 bytes short: refused before anything runs
    with pytest.raises(h.HsmmError) as e:
        h.gemm_grouped(probs, ab, h.R_32F, comp, workspace=ws[:need - 64])
    assert e.value.status == h.hsmm.WORKSPACE_TOO_SMALL


def test_gemm_grouped_captured_in_graph(ora):
    """The whole hsmm_gemm_grouped call (descriptor upload and launch) captured in a CUDA graph
    and replayed: the result is the product, and a second replay after C was overwritten
    writes it again (the graph holds the descriptors; the host array is gone)."""
    h = hsmm()
    probs, hosts = make_problems(SHAPES, 1100, c_aligned=True)
    need = h.gemm_grouped_workspace_size(probs)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    # warm once outside capture (kernel attributes are set on the first launch)
    h.gemm_grouped(probs, workspace=ws, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        h.gemm_grouped(probs, alpha=1.0, beta=0.0, workspace=ws, stream=s)
    for rep in range(2):
        for (_, _, C, _, _) in probs:
            C.fill_(float("nan"))
        ws.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        check(ora, probs, hosts, "N", "N", lambda k: 2 * k * 2.0 ** -24)
