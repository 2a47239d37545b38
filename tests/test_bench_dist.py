"""The benchmark's N > 1 host logic on CPU (no GPU): two ranks over the gloo
backend, as torchrun would start them.  The whole-job figures are the
slowest rank's time and the units all ranks processed; the reference arm
does its work on rank 0 only."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        t, u = bench.aggregate_over_ranks([1.0, 2.5][rank], [10, 20][rank], w)
        # the reference arm: rank 1 returns at once without running the oracle
        ref = None
        if rank == 1:
            class A:
                nx, steps, warmup = 8, 1, 0
            ref = bench.run_reference(A())
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"env": [r, w, local], "t": t, "u": u, "ref": ref}, f)
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_summed_units(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    for rank in range(world):
        d = json.load(open(tmp_path / f"rank{rank}.json"))
        assert d["env"] == [rank, world, rank]
        assert d["t"] == 2.5 and d["u"] == 30.0
        assert d["ref"] is None


def test_one_process_keeps_local_figures():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(1.5, 7, 1) == (1.5, 7.0)
