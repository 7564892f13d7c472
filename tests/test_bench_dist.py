"""bench.py's multi-process path on CPU (gloo, world size 2): the replica
timing takes the slowest rank and sums the elements of all ranks; under a
multi-rank launch only rank 0 runs and prints the reference arm."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        ms, el = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), dist, "cpu")
        out[rank] = (ms, el)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_reduction_gloo():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        assert out[r] == (20.0, 3000.0)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    a = bench.parse()
    assert bench.run_reference(a) == 0
    assert capsys.readouterr().out == ""
