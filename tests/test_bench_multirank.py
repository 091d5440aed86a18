"""The multi-process paths of bench.py on CPU (world size 2, gloo): the replicas' barrier and
max-over-ranks timing, and the reference arm under torchrun (rank 0 alone prints one line)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench._dist_barrier(world)
        v = bench._dist_max(float(10 * rank + 1), world, "cpu")
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
            fh.write(repr(v))
    finally:
        dist.destroy_process_group()


def test_barrier_and_max_over_ranks_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    world = 2
    torch.multiprocessing.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [float(open(tmp_path / f"r{r}.txt").read()) for r in range(world)]
    assert got == [11.0, 11.0]


def test_single_process_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    bench._dist_barrier(1)
    assert bench._dist_max(3.5, 1, "cpu") == 3.5


def test_reference_arm_under_torchrun():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
