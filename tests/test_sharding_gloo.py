"""Multi-rank sharding of the points, run as world-size-2 gloo ranks on CPU.

Each rank evaluates its block of points with the oracle (no GPU here); the
blocks are gathered over gloo and must equal one evaluation of all points.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2004_11571_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, mode, result_path):
    import oracle
    import workloads as wl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = wl.make_zipf(n=6, s=3_000, p=wl.random_prime(62, 3), deg12=8, deg_rest=5, T=21, seed=4)
    if mode == "strong":
        t0, T = sharding.strong_block(w.T, 1, rank, world)
    else:
        t0, T = sharding.weak_block(w.T, 1, rank)
    _, out = oracle.eval_direct(w, T=T, t0=t0)
    rows = torch.from_numpy(out.view(np.int64).copy())
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([rows.shape[0]]))
    mx = int(max(s.item() for s in sizes))
    pad = torch.zeros((mx, rows.shape[1]), dtype=torch.int64)
    pad[: rows.shape[0]] = rows
    gathered = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(gathered, pad)
    if rank == 0:
        full = torch.cat([g[: int(s.item())] for g, s in zip(gathered, sizes)]).numpy()
        total = w.T if mode == "strong" else w.T * world
        _, ref = oracle.eval_direct(w, T=total, t0=1)
        np.save(result_path, np.array([full.shape[0] == total and np.array_equal(full.view(np.uint64), ref)]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["strong", "weak"])
def test_two_gloo_ranks_cover_the_points(mode, tmp_path):
    res = str(tmp_path / "ok.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), mode, res), nprocs=2, join=True, start_method="spawn")
    assert bool(np.load(res)[0])


def test_blocks_partition_the_points():
    for T in (0, 1, 7, 1024):
        for world in (1, 2, 3, 8):
            blocks = [sharding.strong_block(T, 5, r, world) for r in range(world)]
            pts = [t for a, n in blocks for t in range(a, a + n)]
            assert pts == list(range(5, 5 + T))
    assert sharding.weak_block(64, 1, 3) == (193, 64)
    with pytest.raises(ValueError):
        sharding.strong_block(10, 1, 2, 2)
