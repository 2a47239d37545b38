"""One p(l)-CG solve sharded over 2 and 3 gloo ranks on the CPU (the host
model in sharded_model.py: slab halo exchange before every SpMV, the dot
products reduced asynchronously and consumed l iterations later, Algorithm
2's overlap) reproduces the FP64 oracle's iterates x_1, x_2, ... to 1e-12,
for l = 1, 2, 3 and both dot-product variants."""
import os
import socket
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_06850_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
GRID = (10, 9, 12)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    op = W.stencil3d(*GRID)
    b = W.rhs(op, np.random.default_rng(21).standard_normal(W.op_size(op)))
    return op, b


def _rank_main(rank, world, port, out_dir, cases):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path[:0] = [HERE, ROOT]
    import torch.distributed as dist
    import sharded_model as SM
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        op, b = _problem()
        slab = SM.Slab(*GRID, rank, world)
        for l, dots_2l1 in cases:
            sig = [0.5 * 12 + 0.5 * 12 * np.cos((2 * i + 1) * np.pi / (2 * l)) for i in range(l)]
            xs, k, _ = SM.sharded_plcg(slab, op["center"], op["off"], b[slab.rows], l, sig, 1e-10, 500,
                                       dots_2l1=dots_2l1)
            np.save(os.path.join(out_dir, f"r{rank}_l{l}_{int(dots_2l1)}.npy"), np.array(xs))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_model_matches_the_oracle(tmp_path, world):
    mp = pytest.importorskip("torch.multiprocessing")
    cases = [(1, True), (2, True), (3, True), (2, False)]
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), cases), nprocs=world,
                       start_method="spawn", join=True)
    op, b = _problem()
    for l, dots_2l1 in cases:
        parts = [np.load(tmp_path / f"r{r}_l{l}_{int(dots_2l1)}.npy") for r in range(world)]
        assert len({p.shape[0] for p in parts}) == 1          # every rank took the same steps
        xs = np.concatenate(parts, axis=1)                   # x_k for k = 0, 1, ...
        sig = O.chebyshev_shifts(l, 0.0, 12.0)
        final = O.plcg(op, b, l=l, sigma=sig, rtol=1e-10, dots_2l1=dots_2l1)
        assert final.status == O.ORC_OK and xs.shape[0] - 1 == final.iters, (l, xs.shape, final.iters)
        for k in range(1, xs.shape[0]):
            ref = O.plcg(op, b, l=l, sigma=sig, rtol=1e-10, maxit=k, dots_2l1=dots_2l1).x
            err = np.linalg.norm(xs[k] - ref) / np.linalg.norm(ref)
            assert err <= 1e-12, (world, l, dots_2l1, k, err)
