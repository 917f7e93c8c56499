"""The N > 1 launch of bench.py on the CPU: two gloo ranks (replicas only, no data-path collective).

One process per rank as torchrun starts them: the barrier and the max-over-ranks timing reduce
across real ranks, the whole-job value counts every replica's units over the slowest time, and
under two ranks the reference arm runs on rank 0 alone (rank 1 leaves without work or output).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
dist.init_process_group("gloo", rank=rank, world_size=2)
bench.barrier(2)
slowest = bench.max_over_ranks(10.0 + 5.0 * rank, 2)
value = bench.whole_job_value(2, 1.0e9, slowest)
bench.barrier(2)
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "slowest": slowest, "value": value}}))
"""


def launch(code_or_args, port, is_script):
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        cmd = [sys.executable, "-c", code_or_args] if is_script else [sys.executable] + code_or_args
        procs.append(subprocess.Popen(cmd, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_two_gloo_ranks_barrier_and_max_timing():
    outs = launch(WORKER.format(root=ROOT), free_port(), True)
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert [r["rank"] for r in res] == [0, 1]
    for r in res:
        assert r["slowest"] == 15.0                       # the slower rank's time on both ranks
        assert r["value"] == pytest.approx(2 * 1.0e9 / 15e-3)


def test_reference_arm_two_ranks_rank0_only():
    outs = launch(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3", "--size", "384"],
                  free_port(), False)
    line = json.loads(outs[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    for key in ("metric", "value", "unit", "cpu_baseline", "e2e", "config"):
        assert key in line
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert outs[1].strip() == ""                          # rank 1: no work, no output
