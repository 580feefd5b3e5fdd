"""The N > 1 path on CPU (gloo, world size 2).

A single system is not sharded: N GPUs run N independent replicas, so the
only cross-rank steps are the barrier around the timed region and the
max-over-ranks of the step time.  Both are checked here with two gloo ranks,
and the reference arm is launched the way the multi-GPU runs launch it
(torch.distributed.run, 2 processes): rank 0 alone prints its JSON line.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ranks(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sys.path.insert(0, ROOT)
        import bench
        bench.barrier(world)
        m = bench.max_over_ranks(world, float(10 * (rank + 1)), torch.device("cpu"))
        bench.barrier(world)
        out[rank] = m
    finally:
        dist.destroy_process_group()


def test_barrier_and_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_ranks, args=(2, _free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        assert dict(out) == {0: 20.0, 1: 20.0}


def test_reference_arm_two_ranks_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--config", "two_phase_16x16x8"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["higher_is_better"] is False
    assert d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    # the GPU arm prints the same config dict for the same arguments
    sys.path.insert(0, ROOT)
    import bench
    from paper_2101_11649_gb300.synth import CONFIGS

    class A:
        rtol = 1e-8
    assert d["config"] == bench.config_dict(A, "two_phase_16x16x8", CONFIGS["two_phase_16x16x8"]().n, 2)
