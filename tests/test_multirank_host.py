"""The N > 1 host path of bench.py on CPU: two gloo ranks (no GPU).

Each rank solves its own independent problem (the right-hand-side seed is the rank), so the
data path has no collective. Only the timing maximum is all-reduced, and rank 0 alone prints.
These tests run that host logic with world_size 2: the barrier, the max over ranks, and the
reference arm (the oracle on rank 0 only).
"""
import io
import json
import os
import sys
import contextlib

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    m = bench.max_over_ranks(10.0 + rank, world)
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", str(world), "--steps", "1", "--warmup", "0",
                "--n", "16", "--p", "2", "--k", "3"]
    a = bench.parse()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(a, rank, world)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": m, "stdout": buf.getvalue()}, f)


def test_two_gloo_ranks_barrier_max_and_rank0_output(tmp_path):
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["max"] == 11.0 and r1["max"] == 11.0
    assert r1["stdout"] == ""                       # other ranks exit without work or output
    lines = [l for l in r0["stdout"].splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_rank_seeds_give_independent_problems():
    """Weak scaling: rank r solves the right side of seed r, so ranks share no data."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import workloads
    c0 = workloads.random_sine_coeffs(2, seed=0, modes=16)
    c1 = workloads.random_sine_coeffs(2, seed=1, modes=16)
    assert c0.shape == c1.shape and not np.allclose(c0, c1)
