"""Grouped products: one persistent launch for many uneven GEMMs, CUDA-graph replay,
and the autotuner that picks tile widths and the tile schedule.

The tuner's search space (all sweeps within documented limits):
  * tile width per problem: the library's automatic widths (threshold 0: on CTA pairs
    with K-major B, n cut into equal tiles of a multiple of 32 columns), or 256 columns
    when n >= threshold, else 128, for threshold in {129, 193, 257, 385, 513, inf}
    (inf: all 128);
  * schedule: problems in the given order, or longest k first.
Each candidate is built as a plan, launched a few times, timed with CUDA events on
the launching stream, and the fastest is written to a JSON table keyed by a
signature of the problem list, so later runs with the same shapes reuse it.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import hsmm as _h

THRESHOLDS = (0, 129, 193, 257, 385, 513, 1 << 30)
SCHEDULES = (0, 1)
DEFAULT_TABLE = os.path.join(os.path.expanduser("~"), ".cache", "hsmm", "grouped_tune.json")


def signature(problems) -> str:
    """Hash of the (m, n, k, transA, transB, dtype) list."""
    h = hashlib.sha256()
    for A, B, C, ta, tb in problems:
        m, n = C.shape
        k = A.shape[1] if ta.upper() == "N" else A.shape[0]
        h.update(f"{m},{n},{k},{ta},{tb},{A.dtype},{C.dtype};".encode())
    return h.hexdigest()[:24]


def tile_widths(problems, threshold: int):
    """256 columns when n >= threshold, else 128; threshold 0: the library's automatic widths
    (on CTA pairs with K-major B, n cut into equal tiles of a multiple of 32 columns)."""
    if threshold == 0:
        return None
    return [256 if C.shape[1] >= threshold else 128 for (_, _, C, _, _) in problems]


def _dtypes(problems, compute):
    A = problems[0][0]
    C = problems[0][2]
    ab = _h.R_16BF if A.dtype == torch.bfloat16 else _h.R_32F
    c = _h.R_16BF if C.dtype == torch.bfloat16 else _h.R_32F
    if ab == _h.R_32F:
        compute = _h.COMPUTE_32F_FAST_TF32
    return ab, c, compute


def build_plan(problems, threshold=257, schedule=1, compute=_h.COMPUTE_DEFAULT):
    ab, c, compute = _dtypes(problems, compute)
    return _h.GroupedPlan(problems, ab, c, compute, tile_n_per_problem=tile_widths(problems, threshold),
                          schedule=schedule)


def time_plan(plan, reps=10, warmup=3, stream=None) -> float:
    """Mean seconds per launch, CUDA events on the launching stream."""
    stream = stream or torch.cuda.current_stream()
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            plan.launch(stream=stream)
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(reps):
            plan.launch(stream=stream)
        end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / reps * 1e-3


def autotune(problems, compute=_h.COMPUTE_DEFAULT, table_path: str | None = DEFAULT_TABLE, reps=10,
             force=False) -> dict:
    """Time every candidate, keep the fastest; cache the choice in a JSON table."""
    sig = signature(problems)
    table = {}
    if table_path and os.path.exists(table_path):
        try:
            table = json.load(open(table_path))
        except (OSError, ValueError):
            table = {}
    if not force and sig in table:
        return table[sig]
    results = []
    for thr in THRESHOLDS:
        for sched in SCHEDULES:
            plan = build_plan(problems, thr, sched, compute)
            t = time_plan(plan, reps=reps)
            plan.close()
            results.append({"threshold": thr, "schedule": sched, "seconds": t})
    best = min(results, key=lambda r: r["seconds"])
    entry = {"threshold": best["threshold"], "schedule": best["schedule"], "seconds": best["seconds"],
             "candidates": results}
    table[sig] = entry
    if table_path:
        os.makedirs(os.path.dirname(table_path), exist_ok=True)
        tmp = table_path + f".tmp{os.getpid()}"
        json.dump(table, open(tmp, "w"), indent=1)
        os.replace(tmp, table_path)
    return entry


class GroupedGemm:
    """A tuned grouped plan whose single launch is captured once in a CUDA graph."""

    def __init__(self, problems, compute=_h.COMPUTE_DEFAULT, alpha=1.0, beta=0.0, tune=True,
                 table_path: str | None = DEFAULT_TABLE, threshold=257, schedule=1):
        self.problems = list(problems)
        if tune:
            entry = autotune(self.problems, compute, table_path)
            threshold, schedule = entry["threshold"], entry["schedule"]
        self.threshold, self.schedule = threshold, schedule
        self.plan = build_plan(self.problems, threshold, schedule, compute)
        self.alpha, self.beta = alpha, beta
        self.stream = torch.cuda.Stream()
        self.graph = torch.cuda.CUDAGraph()
        # warm once outside capture (first launch sets kernel attributes), then capture
        self.plan.launch(alpha, beta, stream=self.stream)
        self.stream.synchronize()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self.plan.launch(alpha, beta, stream=self.stream)

    def replay(self):
        self.graph.replay()

    def flops(self) -> float:
        tot = 0
        for A, B, C, ta, tb in self.problems:
            m, n = C.shape
            k = A.shape[1] if ta.upper() == "N" else A.shape[0]
            tot += 2 * m * n * k
        return float(tot)
