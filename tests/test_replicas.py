"""Replica runs (bench.py --gpus N): the host logic on CPU with the gloo backend.

The decomposition has no sharded form; N GPUs run N independent replicas and the job's
time is the slowest rank's.  These tests run two gloo ranks on the CPU (no GPU, no NCCL)
and check the max-over-ranks time, the whole-job throughput and that only rank 0 runs the
reference arm.
"""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        assert (w, r) == (world, rank)
        t = bench.max_over_ranks(100.0 + 50.0 * rank, world)  # rank 1 is the slowest
        v = bench.job_throughput(1000, 4, t, world)

        # the reference arm: rank 0 alone runs it; the others return without any work
        calls = []
        bench.oracle_sample = lambda budget, h: calls.append(1) or (1.0, "stub", 0.01)

        class A:
            workload, warmup, steps, cpu_budget, gpus = "er_n2000_h2", 1, 1, 1.0, world

        bench.run_reference(A, world, rank)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{t} {v} {len(calls)}\n")
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    got = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    for r, (t, v, calls) in enumerate(got):
        assert float(t) == 150.0                      # the slowest rank's time on every rank
        assert float(v) == pytest.approx(2 * 1000 * 4 / 0.150)
        assert int(calls) == (2 if r == 0 else 0)     # warmup + steps on rank 0 only


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(10, 2, 1000.0, 1) == 20.0
