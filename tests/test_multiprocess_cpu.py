"""The multi-process path of bench.py on CPU with gloo, world size 2: every rank runs its own replica
(no collective on the data path), the timed region is bracketed by barriers, the reported time is
the max over ranks, and only rank 0 prints. No GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, %r)
import torch.distributed as dist
import bench
world, rank, local = bench.dist_setup("gloo")
bench.barrier(world)
t = bench.max_over_ranks(0.5 + rank, world, "cpu")   # rank 1 is the slower one
bench.barrier(world)
print(json.dumps({"rank": rank, "world": world, "max": t}), flush=True)
dist.destroy_process_group()
"""


def _launch(code, n=2, port=29611, extra_env=None):
    procs = []
    for r in range(n):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(n), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="", **(extra_env or {}))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = [p.communicate(timeout=240) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    return [o for o, _ in outs]


def test_barrier_and_max_over_ranks_with_gloo():
    outs = _launch(WORKER % ROOT)
    recs = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(r["rank"] for r in recs) == [0, 1]
    assert all(r["world"] == 2 and r["max"] == 1.5 for r in recs)


def test_reference_arm_prints_on_rank_0_only():
    code = "import sys; sys.argv=['bench.py','--impl','reference','--steps','1','--warmup','0']; " \
           "sys.path.insert(0, %r); import bench; bench.main()" % ROOT
    outs = _launch(code, port=29612)
    assert outs[1].strip() == ""
    line = json.loads(outs[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["unit"] == "GB/s"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
