"""Host logic of bench.py's N > 1 path, on CPU: two gloo ranks.

bench.py times every rank on its own GPU and reports the slowest rank's time
(a MAX all-reduce of one float, no collective on the data path); under
torchrun only rank 0 prints, and the reference arm runs on rank 0 alone.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(values[rank], dist, "cpu")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world, values = 2, [0.25, 1.5]
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), values, out), nprocs=world, join=True)
    assert [out[r] for r in range(world)] == [max(values)] * world


def test_max_over_ranks_single_process_is_identity():
    assert bench.max_over_ranks(0.125, None, "cpu") == 0.125


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun the reference arm's non-zero ranks do no work and print nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_reference_arm_line_states_what_it_timed():
    """The reference arm's JSON line on the tiny workload: one sampled triplet per step, projected."""
    import json
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "tiny_o6_v36", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["projected"] is True
    assert line["step"] == "one sampled occupied triplet" and line["steps"] == 2
    assert line["config"]["workload"] == "tiny_o6_v36" and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 0 and cb["cores_available"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
