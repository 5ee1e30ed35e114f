"""CPU tests of the benchmark's host logic: the replica (N > 1) aggregation over
torch.distributed with the gloo backend, world size 2, and the reference arm's
behaviour on ranks other than 0 (no work, exit status 0)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [2.0, 3.0][rank]  # rank 1 is the slower replica
        q.put((rank, bench.replica_throughput(local, 10, world, "cpu")))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_is_all_solves_over_the_slowest_rank():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        value, tot = out[r]
        assert tot == 3.0
        assert value == pytest.approx(10 * 2 / 3.0)


def test_single_process_throughput():
    import bench
    assert bench.replica_throughput(4.0, 20, 1, None) == (5.0, 4.0)


def test_reference_arm_other_ranks_do_no_work():
    import argparse
    import bench
    args = argparse.Namespace(gpus=2, steps=3, warmup=3, smoother="chebyshev", mode="mixed")
    assert bench.run_reference(args, 1) == 0
