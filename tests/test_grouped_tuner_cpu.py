"""Host logic of the grouped-launch autotuner (no GPU): candidate widths, the problem-list
signature, the choice of the fastest candidate and its JSON table.  Plans and timings are
replaced by fakes, so only the tuner's own bookkeeping runs."""
import json

import pytest
import torch

from paper_cs_9809105_gb300 import grouped as G


def problems(shapes, dtype=torch.bfloat16, trans=("N", "N")):
    """(A, B, C, transA, transB) with column-major-shaped CPU tensors (only shapes and dtypes are read)."""
    out = []
    for (m, n, k) in shapes:
        A = torch.empty((m, k) if trans[0] == "N" else (k, m), dtype=dtype)
        B = torch.empty((k, n) if trans[1] == "N" else (n, k), dtype=dtype)
        C = torch.empty((m, n), dtype=torch.float32)
        out.append((A, B, C, trans[0], trans[1]))
    return out


SHAPES = [(64, 100, 64), (300, 129, 200), (77, 2048, 33), (1000, 256, 900)]


def test_tile_widths():
    P = problems(SHAPES)
    assert G.tile_widths(P, 0) is None                      # the library's automatic widths
    assert G.tile_widths(P, 129) == [128, 256, 256, 256]
    assert G.tile_widths(P, 257) == [128, 128, 256, 128]
    assert G.tile_widths(P, 1 << 30) == [128] * 4


def test_signature_tracks_shapes_forms_and_dtypes():
    base = G.signature(problems(SHAPES))
    assert base == G.signature(problems(SHAPES))
    assert base != G.signature(problems(SHAPES[::-1]))
    assert base != G.signature(problems(SHAPES, trans=("T", "N")))
    assert base != G.signature(problems(SHAPES, dtype=torch.float32))
    assert base != G.signature(problems(SHAPES[:3] + [(1000, 256, 901)]))


class FakePlan:
    def __init__(self, thr, sched):
        self.key = (thr, sched)
        self.closed = False

    def close(self):
        self.closed = True


@pytest.fixture
def fake_timing(monkeypatch):
    """Every (threshold, schedule) candidate gets a fixed time; (193, 1) is the fastest."""
    built, timed = [], []

    def build_plan(problems, threshold, schedule, compute):
        p = FakePlan(threshold, schedule)
        built.append(p)
        return p

    def time_plan(plan, reps=10, warmup=3, stream=None):
        timed.append(plan.key)
        thr, sched = plan.key
        return 1e-3 + (0 if (thr, sched) == (193, 1) else 1e-4 * (1 + G.THRESHOLDS.index(thr) + sched))

    monkeypatch.setattr(G, "build_plan", build_plan)
    monkeypatch.setattr(G, "time_plan", time_plan)
    return built, timed


def test_autotune_picks_fastest_and_caches(fake_timing, tmp_path):
    built, timed = fake_timing
    table = tmp_path / "tune.json"
    P = problems(SHAPES)
    entry = G.autotune(P, table_path=str(table))
    assert (entry["threshold"], entry["schedule"]) == (193, 1)
    assert len(timed) == len(G.THRESHOLDS) * len(G.SCHEDULES)
    assert all(p.closed for p in built)                        # every candidate plan released
    saved = json.load(open(table))
    assert saved[G.signature(P)]["threshold"] == 193
    # a second call reads the table and times nothing; force re-times
    timed.clear()
    assert G.autotune(P, table_path=str(table)) == saved[G.signature(P)]
    assert timed == []
    G.autotune(P, table_path=str(table), force=True)
    assert len(timed) == len(G.THRESHOLDS) * len(G.SCHEDULES)


def test_autotune_survives_a_broken_table(fake_timing, tmp_path):
    table = tmp_path / "tune.json"
    table.write_text("{not json")
    entry = G.autotune(problems(SHAPES), table_path=str(table))
    assert (entry["threshold"], entry["schedule"]) == (193, 1)
    assert G.signature(problems(SHAPES)) in json.load(open(table))


def test_autotune_without_table(fake_timing):
    _, timed = fake_timing
    entry = G.autotune(problems(SHAPES), table_path=None)
    assert (entry["threshold"], entry["schedule"]) == (193, 1)
    assert len(entry["candidates"]) == len(timed)
