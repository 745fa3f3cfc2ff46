"""Multi-rank sharding, run as world-size-2 gloo ranks on CPU.

Each rank evaluates its share with the oracle (no GPU here): a block of the
points, or a range of (x1, x2) groups (whole output columns); the shares are
gathered over gloo and must equal one evaluation of everything.  Job splits
for batches are checked for balance and coverage.
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


def _group_rank_main(rank, world, port, result_path):
    import oracle
    import workloads as wl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = wl.make_zipf(n=6, s=4_000, p=wl.random_prime(62, 5), deg12=9, deg_rest=5, T=13, seed=6)
    keys, tg = oracle.group_keys(w.exps)
    off = np.concatenate([[0], np.cumsum(np.bincount(tg.astype(np.int64)))])
    g0, g1 = sharding.group_split(off, world)[rank]
    sub = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs[off[g0]:off[g1]], exps=w.exps[off[g0]:off[g1]],
                      beta=w.beta, T=w.T, t0=1)
    _, cols = oracle.eval_direct(sub)                       # this rank's output columns g0..g1-1
    G = keys.shape[0]
    full = torch.zeros((w.T, G), dtype=torch.int64)
    full[:, g0:g1] = torch.from_numpy(cols.view(np.int64).copy())
    dist.all_reduce(full)                                   # disjoint columns: the sum assembles them
    if rank == 0:
        _, ref = oracle.eval_direct(w)
        np.save(result_path, np.array([np.array_equal(full.numpy().view(np.uint64), ref)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_groups(tmp_path):
    res = str(tmp_path / "ok.npy")
    mp.start_processes(_group_rank_main, args=(2, _free_port(), res), nprocs=2, join=True, start_method="spawn")
    assert bool(np.load(res)[0])


def test_group_and_job_splits():
    off = [0, 10, 11, 50, 51, 52, 100]
    for world in (1, 2, 3, 8):
        parts = sharding.group_split(off, world)
        assert parts[0][0] == 0 and parts[-1][1] == 6
        assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
    assert sharding.group_split(off, 2) == [(0, 3), (3, 6)]
    costs = [5.0, 1.0, 9.0, 3.0, 3.0, 7.0, 2.0]
    split = sharding.job_split(costs, 3)
    assert sorted(j for part in split for j in part) == list(range(len(costs)))
    loads = [sum(costs[j] for j in part) for part in split]
    assert max(loads) <= 4 / 3 * max(sum(costs) / 3, max(costs))
    with pytest.raises(ValueError):
        sharding.job_split(costs, 0)
