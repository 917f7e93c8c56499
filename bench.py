"""Benchmark of the hsmm hot path on GB300.

Default workload (one "step"): the FP64-accurate product C = A·B with
m = n = k = 8192 FP64 matrices of entries s·2^e (s ~ U(1,2), random sign,
e ~ U{-12..12}), computed through hsmm_gemm's slice form: error-free splitting of
A (rows) and B (columns) into BF16 slices, the exact slice products on the tcgen05
tensor cores, and the FP64 recombination.  The same JSON line carries the native
FP64 kernel on the same inputs, the error against the accurate (Dot2) product on
256 sampled rows and 4096 sampled entries, the matrix-vector products (16384 x 16384
FP32 and INT8, GB/s), the roofline of the dominant kernel, the CPU oracle baseline,
the SM clocks seen during the timed region, and one sub-object per other workload
(ring: Algorithm 2 at n = 512; autograd: the 4096 x 2048 x 8192 BF16 forward and
backward; grouped: 512 uneven products in one launch; zprecise: the FP64-accurate
complex product), each with its own roofline fraction and a parity line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hsmm|reference]
                  [--workload precise|gemv|autograd|grouped|ring|ring_order|zprecise|nbody|peaks]

Under torchrun (N > 1) every rank runs an independent replica of the step (the
product does not shard without a data-path exchange on one GPU per rank); the
line reports all ranks' flops over the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64-accurate GEMM TFLOP/s vs native FP64 on one GB300 at ≤1e-13 err; GEMV GB/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}

M = N = K = 8192
SLICES, BITS = 7, 7


# ----------------------------------------------------------------------------- helpers
def peaks():
    try:
        p = json.load(open(PEAKS_PATH))
        p["_source"] = "measured"
        return p
    except (OSError, ValueError):
        p = dict(FALLBACK_PEAKS)
        p["_source"] = "fallback"
        return p


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu capture, only while every source file the
    kernel is built from is unchanged (a digest over them is stored beside the figure)."""
    try:
        t = json.load(open(TRAFFIC_PATH))[kernel]
    except (OSError, ValueError, KeyError):
        return None
    srcs = t["sources"] if isinstance(t.get("sources"), list) else [t["source"]]
    import hashlib
    h = hashlib.sha256()
    for rel in srcs:
        path = os.path.join(ROOT, rel)
        if not os.path.exists(path):
            return None
        h.update(open(path, "rb").read())
    if h.hexdigest()[:16] != t["sources_sha"]:
        return None
    return t["bytes_per_launch"]


class ClockSampler:
    """nvidia-smi clock/throttle samples (every 50 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world: int) -> float:
    """The largest of the ranks' values (the job's time is its slowest replica's)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, units_per_rank: float, ms: float) -> float:
    """Whole-job throughput of `world` independent replicas: all units over the slowest time."""
    return world * units_per_rank / (ms / 1e3)


def ev_pair(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# ----------------------------------------------------------------------------- CPU oracle arm
def cpu_oracle_rate(target_seconds: float = 12.0):
    """The oracle's FP64 product (sequential k) on sampled full rows of the 8192^3 workload."""
    import oracle
    import workloads as W
    A, B = W.precise_inputs()
    rows = W.rng(11).choice(M, size=4, replace=False)
    t0 = time.perf_counter()
    oracle.gemm_rows(A, B, rows)
    dt = time.perf_counter() - t0
    nrows = int(max(4, min(M, round(4 * target_seconds / max(dt, 1e-3)))))
    rows = W.rng(12).choice(M, size=nrows, replace=False)
    t0 = time.perf_counter()
    oracle.gemm_rows(A, B, rows)
    dt = time.perf_counter() - t0
    flops = 2.0 * nrows * N * K
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{nrows} full rows of the 8192^3 FP64 product (plain loop, sequential k), {dt:.1f} s"}


def run_reference(args, world, rank):
    """The oracle on the host cores, on a bounded sample of the precise workload; under several
    ranks rank 0 alone runs and prints, the others leave without work."""
    global M, N, K
    if rank != 0:
        return
    import oracle
    import workloads as W
    M = N = K = args.size
    A, B = W.precise_inputs(M, N, K)
    rows = W.rng(11).choice(M, size=2, replace=False)
    t0 = time.perf_counter()
    oracle.gemm_rows(A, B, rows)
    per_row = (time.perf_counter() - t0) / 2
    # each step is a bounded sample: about 4 s of CPU work
    nrows = int(max(1, min(256, round(4.0 / max(per_row, 1e-4)))))
    g = W.rng(13)
    for _ in range(args.warmup):
        oracle.gemm_rows(A, B, g.choice(M, size=nrows, replace=False))
    times = []
    for _ in range(args.steps):
        r = g.choice(M, size=nrows, replace=False)
        t0 = time.perf_counter()
        oracle.gemm_rows(A, B, r)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = 2.0 * nrows * N * K / (ms / 1e3) / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"precise: FP64 C = A*B, m = n = k = {M}, entries s*2^e, e in [-12, 12]",
                       "m": M, "n": N, "k": K, "sample_rows_per_step": nrows},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{nrows} full rows per step of the {M}^3 FP64 product (plain loop)"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
NOMINAL_HBM_GBS = 7900.0       # GB300 HBM3e, nominal
FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64, nominal
NOMINAL_BF16_TFLOPS = 2250.0   # GB300 dense BF16 tensor rate, nominal


def gemv_measure(torch, h, reps=50):
    """Matrix-vector products on the 16384 x 16384 workload: GB/s per form (inputs > L2).

    Each form is also set against two read-only streaming figures: the nominal HBM3e rate
    and a read-only stream measured here on the same 1 GiB matrix (torch's sum reduction,
    a library kernel that reads every byte once); the measured HBM peak in MEASURED_PEAKS.json is a copy
    (read + write), which a read-only stream can exceed."""
    import workloads as W
    out = {}
    m = n = 16384
    A, xs = W.gemv_inputs()
    dA_base = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dA = dA_base.t()
    dx = torch.from_numpy(xs[:n]).cuda()
    dy = torch.zeros(m, device="cuda")
    ws_bytes = max(h.hsmm.gemv_workspace_size(h.R_32F, "N", m, n), h.hsmm.gemv_workspace_size(h.R_8I, "N", m, n))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    A8, x8 = W.gemv_i8_inputs()
    dA8 = torch.from_numpy(np.ascontiguousarray(A8.T)).cuda().t()
    dx8 = torch.from_numpy(x8[:n]).cuda()
    dy8 = torch.zeros(m, dtype=torch.int32, device="cuda")
    del A, A8
    st = torch.cuda.current_stream()
    read_ms = _time_loop(torch, lambda: torch.sum(dA_base), reps, warmup=5)
    read_gbs = m * n * 4 / (read_ms / 1e3) / 1e9
    for name, fn, nbytes in [
        ("f32_N", lambda: h.gemv(dA, dx, dy, "N", workspace=ws), m * n * 4 + (n + m) * 4),
        ("f32_T", lambda: h.gemv(dA, dx, dy, "T", workspace=ws), m * n * 4 + (n + m) * 4),
        ("i8_N", lambda: h.gemv(dA8, dx8, dy8, "N", workspace=ws), m * n + n + 4 * m),
        ("i8_T", lambda: h.gemv(dA8, dx8, dy8, "T", workspace=ws), m * n + n + 4 * m),
    ]:
        for _ in range(5):
            fn()
        s, e = ev_pair(torch)
        s.record(st)
        for _ in range(reps):
            fn()
        e.record(st)
        e.synchronize()
        t = s.elapsed_time(e) / reps * 1e-3
        out[name] = {"GB/s": nbytes / t / 1e9, "us": t * 1e6, "bytes": nbytes}
    return out, read_gbs


def run_precise(args, world, rank, local):
    global M, N, K
    M = N = K = args.size
    import torch
    import paper_cs_9809105_gb300 as h
    from paper_cs_9809105_gb300 import hsmm as H
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pk = peaks()
    A, B = W.precise_inputs(M, N, K)
    # pinned host copies (column-major) for the end-to-end measurement
    hA = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()
    hB = torch.from_numpy(np.ascontiguousarray(B.T)).pin_memory()
    hC = torch.empty((N, M), dtype=torch.float64).pin_memory()
    dA_base = hA.to(dev)
    dB_base = hB.to(dev)
    dA, dB = dA_base.t(), dB_base.t()
    dC = h.colmajor(M, N, torch.float64, dev)
    cfg = H.make_config(h.R_64F, h.R_64F, h.R_64F, h.COMPUTE_64F_OZAKI, SLICES, BITS)
    ws = torch.empty(h.workspace_size(cfg, "N", "N", M, N, K), dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()

    def step():
        h.gemm(dA, dB, dC, compute=h.COMPUTE_64F_OZAKI, slices=SLICES, bits=BITS, workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = h.launch_count()
    with ClockSampler(local) as clk:
        s, e = ev_pair(torch)
        s.record(st)
        for _ in range(args.steps):
            step()
        e.record(st)
        e.synchronize()
    launches = h.launch_count() - launches0
    torch.cuda.synchronize()
    barrier(world)
    ms_local = s.elapsed_time(e) / args.steps
    ms = max_over_ranks(ms_local, world)
    flops = 2.0 * M * N * K
    value = whole_job_value(world, flops, ms) / 1e12
    status = h.sync_status()

    # per-stage kernels, same workload, each timed alone on the launching stream
    # views of the workspace exactly as hsmm_gemm carves it (include/hsmm.h), so the stages
    # below run on the same layout as the timed step
    qa, qb, ea, eb, sd = ozaki_views(torch, ws, M, N, K)
    stages = {}

    def time_stage(name, fn, reps):
        fn()
        torch.cuda.synchronize()
        s1, e1 = ev_pair(torch)
        s1.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        e1.synchronize()
        stages[name] = s1.elapsed_time(e1) / reps
    time_stage("split_A", lambda: h.hsmm.ozaki_split(dA, True, BITS, SLICES, q=qa, expo=ea), 5)
    time_stage("split_B", lambda: h.hsmm.ozaki_split(dB, False, BITS, SLICES, q=qb, expo=eb), 5)
    time_stage("slice_products", lambda: h.hsmm.ozaki_slice_products(qa, qb, K, BITS, sd), args.steps)
    time_stage("recombine", lambda: h.hsmm.ozaki_recombine(sd, ea, eb, dC, BITS), 5)
    pairs = SLICES * (SLICES + 1) // 2
    prod_ms = stages["slice_products"]
    achieved = pairs * flops / (prod_ms / 1e3) / 1e12
    # the slice-product kernel is timed alone (back-to-back launches on the step's workspace):
    # a burst figure, set against the burst peak; the sustained ratio is given beside it
    peak = pk["bf16_tflops"]
    kname = "gemm_ozaki_kernel" if os.environ.get("HSMM_OZAKI_KERNEL") == "single" else "gemm_ozaki_pair_kernel"
    traffic = recorded_traffic(kname)
    roofline = {"kernel": f"{kname} (BF16 slice products, tcgen05)", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"{pk['_source']} bf16 burst (the kernel is timed alone, {args.steps} back-to-back "
                               "launches)",
                "frac_of_sustained": achieved / pk.get("bf16_tflops_sustained", peak),
                "algorithmic": f"{pairs} slice pairs x 2*{M}^3 = {pairs * flops:.4g} flop per launch",
                "traffic": traffic}

    # native FP64 on the same inputs
    dCn = h.colmajor(M, N, torch.float64, dev)
    native = None
    if not args.no_native:
        h.gemm(dA, dB, dCn, compute=h.COMPUTE_64F_NATIVE)
        torch.cuda.synchronize()
        s2, e2 = ev_pair(torch)
        s2.record(st)
        nat_reps = 2
        for _ in range(nat_reps):
            h.gemm(dA, dB, dCn, compute=h.COMPUTE_64F_NATIVE)
        e2.record(st)
        e2.synchronize()
        nat_ms = s2.elapsed_time(e2) / nat_reps
        native = {"value": flops / (nat_ms / 1e3) / 1e12, "unit": "TFLOP/s", "ms": nat_ms,
                  "kernel": "gemm_f64_kernel (FP64 FMA)"}

    # end to end through the public C-ABI call with host buffers (hsmm_gemm_host: H2D of A by
    # row panels and of B by column panels, product by blocks, D2H of every finished block of
    # C, copies overlapped with the product)
    hcfg = H.make_config(h.R_64F, h.R_64F, h.R_64F, h.COMPUTE_64F_OZAKI, SLICES, BITS)
    hws = torch.empty(H.gemm_host_workspace_size(hcfg, "N", "N", M, N, K), dtype=torch.uint8, device=dev)

    def e2e_step():
        h.gemm_host(hA.t(), hB.t(), hC.t(), compute=h.COMPUTE_64F_OZAKI, slices=SLICES, bits=BITS, workspace=hws)

    def e2e_serial_step():
        dA_base.copy_(hA, non_blocking=True)
        dB_base.copy_(hB, non_blocking=True)
        step()
        hC.copy_(dC.t(), non_blocking=True)
    e2e = None
    if not args.no_e2e:
        e2e_reps = max(2, min(args.steps, 5))
        e2e_ms = max_over_ranks(_time_loop(torch, e2e_step, e2e_reps), world)
        serial_ms = _time_loop(torch, e2e_serial_step, e2e_reps)
        e2e = {"value": world * flops / (e2e_ms / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": 2 * M * K * 8, "d2h_bytes_per_step": M * N * 8,
               "api": "hsmm_gemm_host (page-locked host buffers; C in 4 x 2 blocks of 2048 x 4096)",
               "serial_copies_ms_per_step": serial_ms}

    line = None
    if rank == 0:
        # accuracy on sampled rows against the accurate (Dot2) product
        acc = precise_accuracy(torch, A, B, dC, dCn if native is not None else None, dev, args.acc_rows,
                               args.acc_entries)
        gemv, read_gbs = ({}, None) if args.no_gemv else gemv_measure(torch, h)
        for v in gemv.values():
            v["frac_of_nominal_hbm"] = v["GB/s"] / NOMINAL_HBM_GBS
            v["frac_of_read_stream"] = v["GB/s"] / read_gbs
            v["frac_of_measured_copy"] = v["GB/s"] / pk["hbm_gbs"]
        cpu = None if (args.no_cpu_baseline or M != 8192) else cpu_oracle_rate()
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "io_dtype": "f64", "data": "synthetic",
            "config": {"workload": f"precise: FP64-accurate C = A*B, m = n = k = {M}, entries s*2^e, "
                                   "e in [-12, 12]; BF16 slices s = 7 of 7 bits on tcgen05",
                       "m": M, "n": N, "k": K, "slices": SLICES, "bits": BITS,
                       "l2": "inputs larger than L2 (A, B 512 MiB each)"},
            "native_fp64": native, "speedup_vs_native": None if native is None else value / world / native["value"],
            "accuracy": acc, "stages_ms": stages, "roofline": roofline,
            "gemv": {"workload": "16384 x 16384 (FP32 1 GiB / INT8 256 MiB), x of 16384", "forms": gemv,
                     "roofline": None if not gemv else {
                         "kernel": "gemv_f32_n_vec (op = N, FP32)", "bound": "hbm", "achieved": gemv["f32_N"]["GB/s"],
                         "peak": NOMINAL_HBM_GBS, "unit": "GB/s", "frac": gemv["f32_N"]["GB/s"] / NOMINAL_HBM_GBS,
                         "peak_source": "nominal HBM3e rate (a read-only stream may exceed the measured copy, "
                                        f"{pk['hbm_gbs']:.0f} GB/s read + write)",
                         "read_stream_gbs": read_gbs, "measured_copy_gbs": pk["hbm_gbs"],
                         "traffic": recorded_traffic("gemv_f32_n_vec")}},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk.summary(), "status": H.status_string(status),
        }
        if not args.no_extras:
            # the other workloads, each briefly, so that every configuration has a number in the
            # default run (their own --workload modes run them at length)
            extras_reps = 10
            del dA_base, dB_base, dA, dB, ws, hws, dCn, qa, qb, ea, eb, sd
            torch.cuda.empty_cache()
            line["ring"] = measure_ring(torch, h, extras_reps)
            line["autograd"] = measure_autograd(torch, h, extras_reps, pk)
            line["grouped"] = measure_grouped(torch, h, extras_reps, pk, tune=False)
            line["zprecise"] = measure_zprecise(torch, h, 5, pk, 1)
            line["extras_status"] = H.status_string(h.sync_status())
        # the tensor peaks are cuBLAS measurements, which a kernel can pass by a little; far above
        # one would mean the timed kernel does not do the work it is credited with
        line["roofline"]["frac_of_nominal"] = achieved / NOMINAL_BF16_TFLOPS
        frac_max = max([line["roofline"]["frac"]] + [line[k]["roofline"]["frac"] for k in
                                                     ("ring", "autograd", "grouped", "zprecise") if k in line])
        line["roofline_check"] = ("ok" if frac_max <= 1.2 else
                                  f"a fraction of {frac_max:.3f} is far above its measured peak: check the timing")
        print(json.dumps(line), flush=True)
    return line


def ozaki_views(torch, ws, m, n, k):
    """Views of the workspace exactly as hsmm_gemm carves it for the FP64-accurate form
    (include/hsmm.h): slices QA [s][m][kq], QB [s][n][kq], exponents EA, EB, sums SD [s][n][m]."""
    ldq = (k + 7) // 8 * 8
    up = lambda v: (v + 255) // 256 * 256
    pitch = lambda e, z: ((e * z + 255) // 256 * 256 + 1024) // z
    pa, pb, ps = pitch(m * ldq, 2), pitch(n * ldq, 2), pitch(m * n, 4)
    off_qb = up(SLICES * pa * 2)
    off_ea = up(off_qb + SLICES * pb * 2)
    off_eb = up(off_ea + m * 4)
    off_sd = up(off_eb + n * 4)
    qa = ws[:SLICES * pa * 2].view(torch.bfloat16).view(SLICES, pa)[:, :m * ldq].view(SLICES, m, ldq)
    qb = ws[off_qb:off_qb + SLICES * pb * 2].view(torch.bfloat16).view(SLICES, pb)[:, :n * ldq].view(SLICES, n, ldq)
    ea = ws[off_ea:off_ea + 4 * m].view(torch.int32)
    eb = ws[off_eb:off_eb + 4 * n].view(torch.int32)
    sd = ws[off_sd:off_sd + SLICES * ps * 4].view(torch.int32).view(SLICES, ps)[:, :m * n].view(SLICES, n, m)
    return qa, qb, ea, eb, sd


def precise_accuracy(torch, A, B, dC, dCn, dev, nrows, nentries):
    """Error of the FP64-accurate product (and of the native FP64 kernel) against the accurate
    product (Dot2, Ogita-Rump-Oishi) on full sampled rows plus single sampled entries:
    normwise over the sample, the worst row's normwise error, the largest elementwise
    |C - C*| / (|A||B|)_ij and the largest relative error (reported, not bounded: entries
    that cancel make it large)."""
    import oracle
    import workloads as W
    m, k = A.shape
    n = B.shape[1]
    rows = W.rng(21).choice(m, size=min(nrows, m), replace=False)
    ref = oracle.gemm_rows(A, B, rows, accurate=True)
    mag = oracle.gemm_rows(np.abs(A), np.abs(B), rows)
    ridx = torch.from_numpy(rows).to(dev)
    got = dC[ridx].cpu().numpy()
    gotn = dCn[ridx].cpu().numpy() if dCn is not None else None
    row_err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    g = W.rng(22)
    ei = g.integers(0, m, size=nentries)
    ej = g.integers(0, n, size=nentries)
    Bc = [None] * n
    e_ref = np.empty(nentries)
    e_mag = np.empty(nentries)
    for q in range(nentries):
        i, j = int(ei[q]), int(ej[q])
        a_row = np.ascontiguousarray(A[i, :])
        if Bc[j] is None:
            Bc[j] = np.ascontiguousarray(B[:, j])
        e_ref[q] = oracle.dot2(a_row, Bc[j])
        e_mag[q] = float(np.abs(a_row) @ np.abs(Bc[j]))
    e_got = dC[torch.from_numpy(ei).to(dev), torch.from_numpy(ej).to(dev)].cpu().numpy()
    err_all = np.concatenate([np.abs(got - ref).ravel(), np.abs(e_got - e_ref)])
    mag_all = np.concatenate([mag.ravel(), e_mag])
    ref_all = np.concatenate([ref.ravel(), e_ref])
    return {"rows_sampled": int(len(rows)), "entries_sampled": int(nentries),
            "normwise": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "worst_row_normwise": float(row_err.max()),
            "entries_normwise": float(np.linalg.norm(e_got - e_ref) / np.linalg.norm(e_ref)),
            "max_err_over_absA_absB": float(np.max(err_all / mag_all)),
            "max_rel": float(np.max(np.abs(err_all) / np.abs(ref_all))),
            "native_normwise": None if gotn is None else float(np.linalg.norm(gotn - ref) / np.linalg.norm(ref)),
            "bar_normwise": 1e-13,
            "reference": "Dot2 (Ogita-Rump-Oishi) on the host, sampled rows and entries"}


def measure_ring(torch, h, reps):
    """Algorithm 2 on one cluster of p = 16 CTAs, n = 512 FP64, every K dividing 16, against the
    oracle's FP64 triple loop; the integer-valued variant is compared bit for bit."""
    import oracle
    import workloads as W
    n, p = 512, 16
    A, B = W.ring_inputs()
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
    dC = h.colmajor(n, n, torch.float64)
    ms = {}
    for K in (1, 2, 4, 8, 16):
        ws = torch.empty(max(h.hsmm.ring_workspace_size(p, K, n), 16), dtype=torch.uint8, device="cuda")
        ms[K] = _time_loop(torch, lambda: h.ring_gemm(dA, dB, dC, p, K, workspace=ws), reps)
    ws = torch.empty(max(h.hsmm.ring_workspace_size(p, 4, n), 16), dtype=torch.uint8, device="cuda")
    h.ring_gemm(dA, dB, dC, p, 4, workspace=ws)
    torch.cuda.synchronize()
    want = oracle.gemm(A, B)
    mag = oracle.gemm(np.abs(A), np.abs(B))
    gam = n * 2.0 ** -53 / (1 - n * 2.0 ** -53)
    ratio = float(np.max(np.abs(dC.cpu().numpy() - want) / (gam * mag)))
    Ai, Bi = W.ring_inputs(integer=True)
    dAi = torch.from_numpy(np.ascontiguousarray(Ai.T)).cuda().t()
    dBi = torch.from_numpy(np.ascontiguousarray(Bi.T)).cuda().t()
    h.ring_gemm(dAi, dBi, dC, p, 4, workspace=ws)
    torch.cuda.synchronize()
    exact = bool(np.array_equal(dC.cpu().numpy(), oracle.gemm(Ai, Bi)))
    fl = 2.0 * n ** 3
    # the ring runs on the p = 16 SMs of one cluster: their share of the FP64 pipe
    peak = FP64_NOMINAL_TFLOPS * p / 152
    tf = fl / (ms[4] / 1e3) / 1e12
    return {"workload": "ring: C = A B, n = 512 FP64 uniform(-1, 1), p = 16 CTAs (one cluster), b = 32, K = 4",
            "ms": ms[4], "value": tf * 1e3, "unit": "GFLOP/s", "ms_by_K": {str(k): v for k, v in ms.items()},
            "shift_events_by_K": {str(k): (k + p // k - 1 if k > 1 else p - 1) for k in ms},
            "roofline": {"kernel": "ring_kernel (Algorithm 2, FP64)", "bound": "fp64", "achieved": tf,
                         "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "peak_source": f"nominal FP64 rate {FP64_NOMINAL_TFLOPS} TFLOP/s x 16 of 152 SMs"},
            "parity": f"{'ok' if ratio <= 1 and exact else 'FAIL'}: max |C - C*| / (gamma_n |A||B|) = {ratio:.3g}; "
                      f"integer inputs bit-exact: {exact}"}


def measure_autograd(torch, h, reps, pk):
    """C = A B and its backward on the 4096 x 2048 x 8192 BF16 workload: each product timed
    alone, the whole forward + backward step, and sampled rows of C, dA, dB against the oracle."""
    import oracle
    import workloads as W
    from paper_cs_9809105_gb300.autograd import hsmm_matmul
    A_bits, B_bits, G_bits = W.autograd_inputs()
    t = lambda bits: torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    a, b, g = t(A_bits), t(B_bits), t(G_bits)
    m, k = a.shape
    n = b.shape[1]
    fl = 2.0 * m * n * k
    fwd = _time_loop(torch, lambda: h.matmul(a, b, out_dtype=torch.bfloat16), reps)
    da = _time_loop(torch, lambda: h.matmul(g, b, trans_b=True, out_dtype=torch.bfloat16), reps)
    db = _time_loop(torch, lambda: h.matmul(a, g, trans_a=True, out_dtype=torch.bfloat16), reps)
    ar = a.clone().requires_grad_()
    br = b.clone().requires_grad_()

    def step():
        ar.grad = None
        br.grad = None
        hsmm_matmul(ar, br).backward(g)
    step_ms = _time_loop(torch, step, reps)
    # the same forward + backward captured once in a CUDA graph and replayed: the three products
    # without the host work of the eager step (Python binding, autograd engine)
    graphed = {}
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        g_ms = _time_loop(torch, graph.replay, reps)
        graphed = {"ms": g_ms, "TFLOP/s": 3 * fl / (g_ms / 1e3) / 1e12}
    except Exception as e:   # capture refused: reported, the eager figures stand
        graphed = {"unavailable": repr(e)[:200]}
    cub = _time_loop(torch, lambda: a @ b, reps)
    # parity on sampled rows (FP32 outputs), bound k 2^-8 (|.||.|) and the FP32-accumulation bound
    c32 = h.matmul(a, b)
    step()
    torch.cuda.synchronize()
    A64 = np.asfortranarray(W.bf16_bits_to_f64(A_bits))
    B64 = np.asfortranarray(W.bf16_bits_to_f64(B_bits))
    G64 = np.asfortranarray(W.bf16_bits_to_f64(G_bits))
    rr = W.rng(23)
    worst = 0.0
    # FP32 forward: the FP32-accumulation bound 2 k 2^-24; BF16 gradients: that plus one BF16 rounding
    for got_t, X, Y, kk, nrows, rnd in ((c32, A64, B64, k, m, 0.0),
                                        (ar.grad, G64, np.asfortranarray(B64.T), n, m, 2.0 ** -8),
                                        (br.grad, np.asfortranarray(A64.T), G64, m, k, 2.0 ** -8)):
        rows = rr.choice(nrows, size=4, replace=False)
        want = oracle.gemm_rows(X, Y, rows)
        mag = oracle.gemm_rows(np.abs(X), np.abs(Y), rows)
        got = got_t.float()[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        worst = max(worst, float(np.max(np.abs(got - want) / ((2 * kk * 2.0 ** -24 + rnd) * mag + 1e-300))))
    peak = pk["bf16_tflops"]
    per = {"forward_NN": fwd, "dA_NT": da, "dB_TN": db}
    per_gemm = {kk: {"ms": v, "TFLOP/s": fl / (v / 1e3) / 1e12, "frac_of_bf16_burst": fl / (v / 1e3) / 1e12 / peak}
                for kk, v in per.items()}
    slowest = min(x["TFLOP/s"] for x in per_gemm.values())
    return {"workload": "autograd: A 4096x2048, B 2048x8192 BF16 N(0,1/k), dC N(0,1); BF16 out",
            "ms": step_ms, "value": 3 * fl / (step_ms / 1e3) / 1e12, "unit": "TFLOP/s (forward + backward)",
            "per_gemm": per_gemm, "step_in_cuda_graph": graphed,
            "torch_cublas_forward_TFLOP/s": fl / (cub / 1e3) / 1e12,
            "roofline": {"kernel": "gemm_tc_pair_kernel (BF16, 256 x 256 pair tiles), slowest of the three",
                         "bound": "tensor", "achieved": slowest, "peak": peak, "unit": "TFLOP/s",
                         "frac": slowest / peak, "peak_source": f"{pk['_source']} bf16 burst (each product timed alone)"},
            "parity": f"{'ok' if worst <= 1 else 'FAIL'}: C (FP32), dA, dB (BF16) on 4 sampled rows each, max err / "
                      f"((2 k 2^-24 [+ 2^-8 for BF16]) |.||.|) = {worst:.3g}"}


def grouped_problems(torch, shapes, seed):
    """The 512-problem batching workload on the device: BF16 uniform(-1, 1), FP32 C, every
    leading dimension padded to 8 elements."""
    import workloads as W
    g = torch.Generator(device="cuda").manual_seed(seed)
    probs = []
    for (m, n, k) in shapes:
        lda = W.pad_ld(m); ldb = W.pad_ld(k)
        A = (torch.rand((k, lda), generator=g, device="cuda") * 2 - 1).to(torch.bfloat16).t()[:m]
        B = (torch.rand((n, ldb), generator=g, device="cuda") * 2 - 1).to(torch.bfloat16).t()[:k]
        C = torch.empty((n, W.pad_ld(m)), device="cuda").t()[:m]
        probs.append((A, B, C, "N", "N"))
    return probs


def measure_grouped(torch, h, reps, pk, tune=False):
    """512 uneven BF16 products: one persistent launch replayed from a CUDA graph, against 512
    separate launches; sampled rows of sampled problems against the oracle."""
    import oracle
    import workloads as W
    from paper_cs_9809105_gb300.grouped import GroupedGemm
    shapes = [tuple(int(v) for v in sh) for sh in W.grouped_shapes()]
    probs = grouped_problems(torch, shapes, W.SEED_GROUPED)
    # without tuning: the automatic tile widths (threshold 0) and longest-k-first schedule the
    # tuner picks on this problem set
    gg = GroupedGemm(probs, tune=tune, table_path=None, threshold=0, schedule=1)
    flops = gg.flops()
    ms_graph = _time_loop(torch, gg.replay, reps)
    # the same plan on the one-CTA kernel (128-row tiles), for comparison
    os.environ["HSMM_GROUPED_KERNEL"] = "single"
    try:
        gs = GroupedGemm(probs, tune=False, table_path=None, threshold=gg.threshold, schedule=gg.schedule)
        ms_single = _time_loop(torch, gs.replay, reps)
        del gs
    finally:
        del os.environ["HSMM_GROUPED_KERNEL"]

    def loop():
        for (A, B, C, ta, tb) in probs:
            h.gemm(A, B, C, ta, tb)
    ms_loop = _time_loop(torch, loop, 2, warmup=1)
    gg.replay()
    torch.cuda.synchronize()
    rr = W.rng(24)
    worst = 0.0
    for q in rr.choice(len(probs), size=16, replace=False):
        A, B, C, _, _ = probs[int(q)]
        A64 = np.asfortranarray(A.float().double().cpu().numpy())
        B64 = np.asfortranarray(B.float().double().cpu().numpy())
        rows = rr.choice(A64.shape[0], size=min(4, A64.shape[0]), replace=False)
        want = oracle.gemm_rows(A64, B64, rows)
        mag = oracle.gemm_rows(np.abs(A64), np.abs(B64), rows)
        got = C[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        worst = max(worst, float(np.max(np.abs(got - want) / (2 * A64.shape[1] * 2.0 ** -24 * mag + 1e-300))))
    gbytes = sum(m * k * 2 + k * n * 2 + m * n * 4 for (m, n, k) in shapes) / 1e9
    gbs = gbytes / (ms_graph / 1e3)
    tuned = {"threshold": gg.threshold, "schedule": gg.schedule}
    del gg, probs
    tf32 = measure_grouped_tf32(torch, h, reps, pk, shapes)
    return {"workload": "grouped: 512 problems, m, n, k log-uniform in [64, 2048], BF16, FP32 C, ld padded to 8",
            "ms": ms_graph, "value": flops / (ms_graph / 1e3) / 1e12, "unit": "TFLOP/s",
            "total_flop": flops, "tuned": tuned,
            "loop_of_512_launches": {"ms": ms_loop, "TFLOP/s": flops / (ms_loop / 1e3) / 1e12},
            "speedup_vs_loop": ms_loop / ms_graph,
            "one_cta_tiles_ms": ms_single,
            # A and B read once, C written once (FP32): on these shapes the bytes outweigh the flops
            "roofline": {"kernel": "gemm_grouped_pair_kernel<bf16> (256-row tiles on CTA pairs)", "bound": "hbm",
                         "achieved": gbs,
                         "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
                         "algorithmic_bytes": gbytes * 1e9, "traffic": recorded_traffic("gemm_grouped_pair_kernel"),
                         "tensor_time_at_peak_ms": flops / (pk["bf16_tflops"] * 1e12) * 1e3,
                         "hbm_time_at_peak_ms": gbytes / pk["hbm_gbs"] * 1e3,
                         "peak_source": f"{pk['_source']} HBM copy (read + write, like A, B in and C out)"},
            "parity": f"{'ok' if worst <= 1 else 'FAIL'}: 16 problems x 4 rows, max err / (2 k 2^-24 |A||B|) = "
                      f"{worst:.3g}",
            "tf32": tf32}


def measure_grouped_tf32(torch, h, reps, pk, shapes):
    """The FP32/TF32 variant of the batching workload: the same 512 shapes with FP32 A, B
    (uniform(-1, 1), leading dimensions padded to 4) and FP32 C, TF32 tensor-core products,
    one launch from a CUDA graph; sampled rows against the oracle at the TF32 bound."""
    import oracle
    import workloads as W
    from paper_cs_9809105_gb300.grouped import GroupedGemm
    g = torch.Generator(device="cuda").manual_seed(W.SEED_GROUPED + 1)
    probs = []
    for (m, n, k) in shapes:
        A = (torch.rand((k, W.pad_ld(m, 4)), generator=g, device="cuda") * 2 - 1).t()[:m]
        B = (torch.rand((n, W.pad_ld(k, 4)), generator=g, device="cuda") * 2 - 1).t()[:k]
        C = torch.empty((n, W.pad_ld(m, 4)), device="cuda").t()[:m]
        probs.append((A, B, C, "N", "N"))
    gg = GroupedGemm(probs, tune=False, table_path=None, threshold=0, schedule=1)
    flops = gg.flops()
    ms = _time_loop(torch, gg.replay, reps)
    gg.replay()
    torch.cuda.synchronize()
    rr = W.rng(25)
    worst = 0.0
    for q in rr.choice(len(probs), size=8, replace=False):
        A, B, C, _, _ = probs[int(q)]
        A64 = np.asfortranarray(A.double().cpu().numpy())
        B64 = np.asfortranarray(B.double().cpu().numpy())
        rows = rr.choice(A64.shape[0], size=min(4, A64.shape[0]), replace=False)
        want = oracle.gemm_rows(A64, B64, rows)
        mag = oracle.gemm_rows(np.abs(A64), np.abs(B64), rows)
        got = C[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        kk = A64.shape[1]
        # TF32 keeps 10 fraction bits of each input (|d(ab)| <= 2^-9 |a||b|), plus FP32 sums
        worst = max(worst, float(np.max(np.abs(got - want) / ((2.0 ** -9 + kk * 2.0 ** -23) * mag + 1e-300))))
    gbytes = sum(m * k * 4 + k * n * 4 + m * n * 4 for (m, n, k) in shapes) / 1e9
    gbs = gbytes / (ms / 1e3)
    del gg, probs
    return {"workload": "the same 512 shapes, FP32 A, B and C, TF32 products, ld padded to 4", "ms": ms,
            "TFLOP/s": flops / (ms / 1e3) / 1e12, "GB/s": gbs, "frac_of_measured_copy": gbs / pk["hbm_gbs"],
            "parity": f"{'ok' if worst <= 1 else 'FAIL'}: 8 problems x 4 rows, max err / ((2^-9 + k 2^-23) |A||B|) = "
                      f"{worst:.3g}"}


def measure_zprecise(torch, h, reps, pk, world, size=4096, native=True):
    """FP64-accurate complex product (Section 7 measures complex data) through the real form
    A' B'' (m x 2n x 2k on the slice kernels) against the complex FP64-pipe kernel; normwise
    error on sampled rows against the accurate product."""
    import oracle
    import workloads as W
    from paper_cs_9809105_gb300 import hsmm as H
    m = n = k = size
    A, B = W.zprecise_inputs(m, n, k)
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
    dC = h.colmajor(m, n, torch.complex128)
    cfg = H.make_config(h.C_64F, h.C_64F, h.C_64F, h.COMPUTE_64F_OZAKI, SLICES, BITS)
    ws = torch.empty(h.workspace_size(cfg, "N", "N", m, n, k), dtype=torch.uint8, device="cuda")
    step = lambda: h.gemm(dA, dB, dC, compute=h.COMPUTE_64F_OZAKI, slices=SLICES, bits=BITS, workspace=ws)
    ms = _time_loop(torch, step, reps)
    flops = 8.0 * m * n * k
    pairs = SLICES * (SLICES + 1) // 2
    # the slice products of the real form alone (m x 2n x 2k) on the slices the step left in the
    # workspace, for the roofline; then the step once more, so C is the step's result
    qa, qb, _, _, sd = ozaki_views(torch, ws, m, 2 * n, 2 * k)
    sp_ms = _time_loop(torch, lambda: H.ozaki_slice_products(qa, qb, 2 * k, BITS, sd), reps)
    achieved = pairs * 2.0 * m * (2 * n) * (2 * k) / (sp_ms / 1e3) / 1e12
    nat_ms = None
    if native:
        dCn = h.colmajor(m, n, torch.complex128)
        nat_ms = _time_loop(torch, lambda: h.gemm(dA, dB, dCn, compute=h.COMPUTE_64F_NATIVE), 1, warmup=1)
    step()
    torch.cuda.synchronize()
    rows = W.rng(22).choice(m, size=8, replace=False)
    ref = oracle.zgemm_rows(A, B, rows)
    got = dC[torch.from_numpy(rows).cuda()].cpu().numpy()
    nw = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    out = {"workload": f"zprecise: FP64-accurate complex C = A B, m = n = k = {m}, real and imaginary parts s*2^e, "
                       "e in [-12, 12]; real form m x 2n x 2k, BF16 slices s = 7 of 7 bits",
           "ms": ms, "value": world * flops / (ms / 1e3) / 1e12, "unit": "TFLOP/s (8mnk real flops)",
           "roofline": {"kernel": "gemm_ozaki_pair_kernel (slice products of the real form)", "bound": "tensor",
                        "achieved": achieved, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                        "frac": achieved / pk["bf16_tflops"], "slice_products_ms": sp_ms,
                        "peak_source": f"{pk['_source']} bf16 burst (kernel timed alone)"},
           "accuracy": {"rows_sampled": 8, "normwise": nw, "bar_normwise": 1e-13},
           "parity": f"{'ok' if nw <= 1e-13 else 'FAIL'}: normwise {nw:.3g} against Dot2 on 8 sampled rows"}
    if nat_ms is not None:
        out["native_complex_fp64"] = {"ms": nat_ms, "TFLOP/s": flops / (nat_ms / 1e3) / 1e12,
                                      "kernel": "gemm_z64_kernel (FP64 FMA)"}
        out["speedup_vs_native"] = nat_ms / ms
    return out


def run_zprecise(args, world, rank, local):
    """Complex product (Section 7: the method on complex data), FP64-accurate through the real
    form A' B'' (m x 2n x 2k on the slice kernels) against the complex FP64-pipe kernel, plus the
    end-to-end rate through hsmm_gemm_host with page-locked host buffers."""
    import torch
    import paper_cs_9809105_gb300 as h
    from paper_cs_9809105_gb300 import hsmm as H
    import workloads as W
    torch.cuda.set_device(local)
    pk = peaks()
    m = n = k = args.size if args.size != 8192 else 4096
    launches0 = h.launch_count()
    res = measure_zprecise(torch, h, args.steps, pk, world, size=m)
    launches = h.launch_count() - launches0
    A, B = W.zprecise_inputs(m, n, k)
    hA = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()
    hB = torch.from_numpy(np.ascontiguousarray(B.T)).pin_memory()
    hC = torch.empty((n, m), dtype=torch.complex128).pin_memory()
    cfg = H.make_config(h.C_64F, h.C_64F, h.C_64F, h.COMPUTE_64F_OZAKI, SLICES, BITS)
    hws = torch.empty(H.gemm_host_workspace_size(cfg, "N", "N", m, n, k), dtype=torch.uint8, device="cuda")

    def e2e_step():
        h.gemm_host(hA.t(), hB.t(), hC.t(), compute=h.COMPUTE_64F_OZAKI, slices=SLICES, bits=BITS, workspace=hws)
    e2e_ms = max_over_ranks(_time_loop(torch, e2e_step, max(2, min(args.steps, 5))), world)
    ms = max_over_ranks(res["ms"], world)
    flops = 8.0 * m * n * k
    status = h.sync_status()
    if rank == 0:
        line = {"metric": "FP64-accurate complex GEMM TFLOP/s (8mnk real flops) vs native complex FP64",
                "value": world * flops / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "io_dtype": "c128", "data": "synthetic",
                "config": {"workload": res["workload"], "l2": "inputs larger than L2 (A, B 256 MiB each)"},
                "e2e": {"value": world * flops / (e2e_ms / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                        "h2d_bytes_per_step": 2 * m * k * 16, "d2h_bytes_per_step": m * n * 16},
                "gpu_launches": int(launches), "status": H.status_string(status)}
        for key in ("roofline", "accuracy", "parity", "native_complex_fp64", "speedup_vs_native"):
            if key in res:
                line[key] = res[key]
        print(json.dumps(line), flush=True)


def run_nbody(args, world, rank, local):
    """The two-array n^2 problem of Section 4 (gravitational instance, Section 2): tiled schedule
    against the hyper-systolic recipe with regular bases on thread-block clusters."""
    import torch
    import paper_cs_9809105_gb300 as h
    from paper_cs_9809105_gb300 import hsmm as H
    import workloads as W
    torch.cuda.set_device(local)
    pk = peaks()
    x = torch.from_numpy(W.nbody_bodies().astype(np.float32)).cuda()
    n = x.shape[0]
    out = torch.empty_like(x)
    inter = float(n) * n
    tiled_ms = _time_loop(torch, lambda: h.nbody(x, x, W.NBODY_EPS2, out), args.steps, warmup=args.warmup)
    hs = {}
    for p, K in ((4, 1), (4, 2), (4, 4), (8, 2), (8, 4), (16, 2), (16, 4)):
        try:
            ms = _time_loop(torch, lambda: h.nbody(x, x, W.NBODY_EPS2, out, ring_p=p, ring_k=K), args.steps)
        except h.HsmmError as e:
            hs[f"p{p}_K{K}"] = {"unavailable": str(e)}
            continue
        hs[f"p{p}_K{K}"] = {"ms": ms, "G_interactions/s": inter / (ms / 1e3) / 1e9,
                            "shift_events_per_round": 2 * K + p // K - 3}
    status = h.sync_status()
    if rank == 0:
        value = world * inter / (tiled_ms / 1e3) / 1e9
        # FP32 lane operations per interaction, counted from the kernel: 3 subtractions, 3 FMAs
        # for r^2, 2 multiplications for inv^3, 1 for the mass, 3 FMAs into a (plus one reciprocal
        # square root on the special-function unit); eps2 > 0 needs no select for r = 0
        ops = 12
        lanes = 152 * 128
        peak_ops = lanes * pk.get("sm_max_mhz", 2070) * 1e6 / 1e12          # T lane-ops/s
        achieved = inter * ops / (tiled_ms / 1e3) / 1e12
        print(json.dumps({
            "metric": "two-array n^2 problem (gravitational n-body), G interactions/s", "value": value,
            "unit": "G interactions/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tiled_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"nbody: {n} bodies uniform in the unit ball, masses U(0.5, 1.5)/n, eps2 = "
                                   f"{W.NBODY_EPS2}, all n^2 pairs"},
            "tflops_at_20_flop_per_interaction": value * 20 / 1e3,
            "hyper_systolic": hs,
            "roofline": {"kernel": "nbody_tiled", "bound": "alu", "achieved": achieved, "peak": peak_ops,
                         "unit": "T FP32 lane-ops/s", "frac": achieved / peak_ops,
                         "peak_source": "152 SMs x 128 FP32 lanes x max SM clock (measured peaks file)",
                         "ops_per_interaction": ops},
            "status": H.status_string(status), "gpu_launches": 1}), flush=True)


def run_gemv(args, world, rank, local):
    import torch
    import paper_cs_9809105_gb300 as h
    torch.cuda.set_device(local)
    pk = peaks()
    out, read_gbs = gemv_measure(torch, h, reps=max(args.steps, 20))
    if rank == 0:
        v = out["f32_N"]["GB/s"]
        print(json.dumps({"metric": "GEMV GB/s (16384 x 16384 FP32, y = A x)", "value": v * world, "unit": "GB/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": "gemv 16384 x 16384"}, "forms": out,
                          "roofline": {"bound": "hbm", "achieved": v, "peak": NOMINAL_HBM_GBS, "unit": "GB/s",
                                       "frac": v / NOMINAL_HBM_GBS, "peak_source": "nominal HBM3e rate",
                                       "read_stream_gbs": read_gbs, "measured_copy_gbs": pk["hbm_gbs"],
                                       "traffic": recorded_traffic("gemv_f32_n_vec")}}),
              flush=True)


def _time_loop(torch, fn, reps, warmup=3, stream=None):
    st = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s, e = ev_pair(torch)
    s.record(st)
    for _ in range(reps):
        fn()
    e.record(st)
    e.synchronize()
    return s.elapsed_time(e) / reps


def run_autograd(args, world, rank, local):
    """Differentiation form: C = A B (4096 x 2048 x 8192 BF16, FP32 accumulation), dA = dC B^T, dB = A^T dC."""
    import torch
    import paper_cs_9809105_gb300 as h
    torch.cuda.set_device(local)
    pk = peaks()
    launches0 = h.launch_count()
    res = measure_autograd(torch, h, args.steps, pk)
    launches = h.launch_count() - launches0
    if rank == 0:
        print(json.dumps({
            "metric": "autograd C = A B + backward, TFLOP/s (BF16, FP32 accumulation)", "value": res["value"],
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": res["workload"]}, "per_gemm": res["per_gemm"],
            "step_in_cuda_graph": res["step_in_cuda_graph"],
            "torch_cublas_forward_TFLOP/s": res["torch_cublas_forward_TFLOP/s"], "roofline": res["roofline"],
            "parity": res["parity"], "gpu_launches": int(launches)}), flush=True)


def run_grouped(args, world, rank, local):
    """Batching form: 512 products, m, n, k log-uniform in [64, 2048], BF16, one persistent launch in a graph."""
    import torch
    import paper_cs_9809105_gb300 as h
    torch.cuda.set_device(local)
    pk = peaks()
    res = measure_grouped(torch, h, args.steps, pk, tune=not args.no_tune)
    if rank == 0:
        print(json.dumps({
            "metric": "grouped GEMM aggregate TFLOP/s (512 problems, BF16, one launch in a CUDA graph)",
            "value": res["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": res["workload"], "total_flop": res["total_flop"], "tuned": res["tuned"]},
            "loop_of_512_launches": res["loop_of_512_launches"], "speedup_vs_loop": res["speedup_vs_loop"],
            "roofline": res["roofline"], "parity": res["parity"], "tf32": res["tf32"], "gpu_launches": 1}), flush=True)


def run_ring(args, world, rank, local):
    """The paper's Algorithm 2: n = 512 FP64, p = 16 CTAs in one cluster, K = 4 (every K dividing 16 beside it)."""
    import torch
    import paper_cs_9809105_gb300 as h
    torch.cuda.set_device(local)
    res = measure_ring(torch, h, args.steps)
    if rank == 0:
        print(json.dumps({
            "metric": "hyper-systolic ring product (Algorithm 2), GFLOP/s, n = 512 FP64, p = 16",
            "value": res["value"], "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": res["workload"]},
            "ms_by_K": res["ms_by_K"], "shift_events_by_K": res["shift_events_by_K"], "roofline": res["roofline"],
            "parity": res["parity"], "gpu_launches": 1}), flush=True)


def run_ring_order(args, world, rank, local):
    """Tile reuse order of the tensor-core product: persistent tiles (operands from L2) against
    the ring order of Algorithm 2 on thread-block clusters (A blocks passed between CTAs
    through distributed shared memory, K auxiliary accumulators in TMEM), BF16 8192^3."""
    import torch
    import paper_cs_9809105_gb300 as h
    import workloads as W
    torch.cuda.set_device(local)
    m = n = k = args.size
    dA = W_dev_bf16(torch, W.uniform_bf16((m, k), 920))
    dB = W_dev_bf16(torch, W.uniform_bf16((k, n), 921))
    dC = h.colmajor(m, n, torch.float32)
    fl = 2.0 * m * n * k
    tf = lambda ms: fl / (ms / 1e3) / 1e12
    persistent = {
        "pair 256x256 (cta_group::2)": _time_loop(torch, lambda: h.gemm(dA, dB, dC), args.steps),
        "single CTA 128x128": _time_loop(torch, lambda: h.gemm(dA, dB, dC, tile_n=128), args.steps),
    }
    os.environ["HSMM_GEMM_KERNEL"] = "single"
    persistent["single CTA 128x256"] = _time_loop(torch, lambda: h.gemm(dA, dB, dC, tile_n=256), args.steps)
    del os.environ["HSMM_GEMM_KERNEL"]
    ring = {}
    for p, K in ((2, 1), (2, 2), (4, 1), (4, 2), (4, 4), (8, 1), (8, 2), (8, 4), (16, 2), (16, 4)):
        try:
            ms = _time_loop(torch, lambda: h.gemm(dA, dB, dC, ring_p=p, ring_k=K), args.steps)
        except h.HsmmError as e:
            ring[f"p{p}_K{K}"] = {"unavailable": str(e)}
            continue
        panels, rows = -(-n // (128 * p)), -(-m // 128)
        rounds = -(-(-(-k // 64)) // p)
        ctas = panels * p * rows
        ring[f"p{p}_K{K}"] = {
            "ms": ms, "TFLOP/s": tf(ms),
            # A blocks forwarded through DSMEM: K~ - 1 per CTA and round; C blocks back-shifted: K - 1 per CTA
            "dsmem_bytes": ctas * (rounds * (p // K - 1) * 16384 + (K - 1) * 65536),
            # operand blocks loaded by TMA: one A block per CTA and round, p B blocks per CTA and round
            "tma_bytes": ctas * rounds * (1 + p) * 16384}
    status = h.sync_status()
    best = max((v["TFLOP/s"] for v in ring.values() if "TFLOP/s" in v), default=None)
    if rank == 0:
        print(json.dumps({
            "metric": "BF16 GEMM TFLOP/s by tile reuse order (persistent vs ring order of Algorithm 2)",
            "value": best, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"ring_order: C = A B, m = n = k = {m}, BF16 uniform(-1,1), FP32 out",
                       "l2": "inputs larger than L2 (A, B, C 128 + 128 + 256 MiB)"},
            "persistent": {kname: {"ms": v, "TFLOP/s": tf(v)} for kname, v in persistent.items()},
            "ring_order": ring, "status": h.hsmm.status_string(status),
            "gpu_launches": 1}), flush=True)


def W_dev_bf16(torch, bits):
    """Column-major BF16 device matrix from 16-bit patterns."""
    t = torch.from_numpy(np.ascontiguousarray(bits.T).view(np.int16)).cuda()
    return t.view(torch.bfloat16).t()


def run_peaks(args, world, rank, local):
    """Rates of the arithmetic pipes the peak file does not hold (TF32, INT8 and FP64 through
    cuBLAS via torch), beside this library's own TF32, BF16 and FP64 kernels on the same shapes:
    the denominators for the TF32 and FP64 rows and the evidence for taking BF16 slices."""
    import torch
    import paper_cs_9809105_gb300 as h
    torch.cuda.set_device(local)
    g = torch.Generator(device="cuda").manual_seed(7)
    out = {}

    def rate(fn, flops, reps):
        return flops / (_time_loop(torch, fn, reps) / 1e3) / 1e12

    n = args.size
    a32 = torch.rand(n, n, device="cuda", generator=g) - 0.5
    b32 = torch.rand(n, n, device="cuda", generator=g) - 0.5
    c32 = torch.empty(n, n, device="cuda")
    fl = 2.0 * n ** 3
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    out["cublas_tf32_tflops"] = rate(lambda: torch.mm(a32, b32, out=c32), fl, 10)
    torch.backends.cuda.matmul.allow_tf32 = prev
    ct = h.colmajor(n, n, torch.float32)
    out["hsmm_tf32_tflops"] = rate(lambda: h.gemm(a32.t(), b32.t(), ct, "T", "N", compute=h.COMPUTE_32F_FAST_TF32),
                                   fl, 10)   # TF32: K-major forms
    ab, bb = a32.to(torch.bfloat16), b32.to(torch.bfloat16)
    out["cublas_bf16_tflops"] = rate(lambda: torch.mm(ab, bb), fl, 10)
    out["hsmm_bf16_tflops"] = rate(lambda: h.gemm(ab.t(), bb.t(), ct, "T", "N"), fl, 10)
    del a32, b32, c32, ct, ab, bb
    a8 = torch.randint(-128, 128, (n, n), device="cuda", generator=g, dtype=torch.int8)
    b8 = torch.randint(-128, 128, (n, n), device="cuda", generator=g, dtype=torch.int8)
    try:
        out["cublas_int8_tops"] = rate(lambda: torch._int_mm(a8, b8), fl, 10)
    except RuntimeError as e:
        out["cublas_int8_tops"] = None
        out["cublas_int8_error"] = str(e).splitlines()[0][:200]
    del a8, b8
    n = args.size // 2
    a64 = torch.rand(n, n, device="cuda", generator=g, dtype=torch.float64)
    b64 = torch.rand(n, n, device="cuda", generator=g, dtype=torch.float64)
    c64 = h.colmajor(n, n, torch.float64)
    fl = 2.0 * n ** 3
    out["cublas_fp64_tflops"] = rate(lambda: torch.mm(a64, b64), fl, 3)
    out["hsmm_fp64_tflops"] = rate(lambda: h.gemm(a64.t(), b64.t(), c64, compute=h.COMPUTE_64F_NATIVE), fl, 3)
    if rank == 0:
        print(json.dumps({"metric": "arithmetic pipe rates (dense products, TFLOP/s or TOP/s)",
                          "config": {"workload": f"peaks: {args.size}^3 TF32, BF16, INT8 and {args.size // 2}^3 FP64 "
                                                 "products, uniform inputs"},
                          "rates": out, "clocks": None}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hsmm", choices=["hsmm", "reference"])
    ap.add_argument("--workload", default="precise", choices=["precise", "gemv", "autograd", "grouped", "ring",
                                                               "ring_order", "zprecise", "nbody", "peaks"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gemv", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="precise workload: leave out the host-buffer measurement")
    ap.add_argument("--no-native", action="store_true", help="precise workload: leave out the native FP64 kernel")
    ap.add_argument("--no-extras", action="store_true",
                    help="precise workload: leave out the ring, autograd, grouped and complex sub-measurements")
    ap.add_argument("--acc-rows", type=int, default=256, help="precise workload: full rows checked against Dot2")
    ap.add_argument("--acc-entries", type=int, default=4096, help="precise workload: single entries checked")
    ap.add_argument("--no-tune", action="store_true", help="grouped workload: skip the autotuner")
    ap.add_argument("--size", type=int, default=8192,
                    help="m = n = k of the precise workload (peaks: of the TF32, BF16 and INT8 products; FP64 half)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        import paper_cs_9809105_gb300 as h
        h.lib()
    except RuntimeError:
        import __graft_entry__
        __graft_entry__.build()
    {"precise": run_precise, "gemv": run_gemv, "autograd": run_autograd, "grouped": run_grouped,
     "ring": run_ring, "ring_order": run_ring_order,
     "zprecise": run_zprecise, "nbody": run_nbody, "peaks": run_peaks}[args.workload](args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
