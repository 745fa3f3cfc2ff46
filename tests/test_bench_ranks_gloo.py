"""The benchmark's multi-rank logic on two gloo ranks (CPU).

bench.py under torchrun gives each rank a share of the workload (rank_share:
weak, strong or group split) and reports the whole job's throughput as the
term-points of every rank over the slowest rank's time (reduce_over_ranks).
Here each rank evaluates its share with the oracle; the shares gathered on
rank 0 must be exactly one evaluation of the whole workload (weak: twice the
points), and the reductions must give the max and the sum over ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    return port


def _gather_rows(arr, world):
    t = torch.from_numpy(np.ascontiguousarray(arr).view(np.int64).reshape(-1).copy())
    n = torch.tensor([t.numel()], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n)
    m = int(max(x.item() for x in sizes))
    pad = torch.zeros(m, dtype=torch.int64)
    pad[:t.numel()] = t
    parts = [torch.zeros(m, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, pad)
    return [p[:int(sz.item())].numpy().view(np.uint64) for p, sz in zip(parts, sizes)]


def _rank_main(rank, world, port, result_path):
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import workloads as wl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ok = []
    w = wl.make_zipf(n=6, s=4_000, p=wl.random_prime(62, 3), deg12=9, deg_rest=5, T=19, seed=4)
    keys, full = oracle.eval_direct(w)
    for split in ("weak", "strong", "group"):
        sub, t0, T, scaling = bench.rank_share(w, split, rank, world)
        sk, img = oracle.eval_direct(sub, T=T, t0=t0)
        parts = _gather_rows(img, world)
        kparts = _gather_rows(sk.astype(np.uint64), world)
        if rank == 0:
            if split == "weak":
                _, both = oracle.eval_direct(w, T=world * w.T, t0=w.t0)
                got = np.concatenate([p.reshape(-1, full.shape[1]) for p in parts])
                ok.append(scaling == "weak" and np.array_equal(got, both))
            elif split == "strong":
                got = np.concatenate([p.reshape(-1, full.shape[1]) for p in parts])
                ok.append(scaling == "strong" and np.array_equal(got, full))
            else:
                cols = [p.reshape(w.T, -1) for p in parts]
                ks = np.concatenate([k.reshape(-1, 2) for k in kparts]).astype(np.uint32)
                ok.append(scaling == "strong" and np.array_equal(np.concatenate(cols, axis=1), full)
                          and np.array_equal(ks, keys) and all(c.shape[1] > 0 for c in cols))
    mx = bench.reduce_over_ranks([1.5 + rank, -rank], dist, "cpu", "max")
    sm = bench.reduce_over_ranks([1.5 + rank, 10.0], dist, "cpu", "sum")
    if rank == 0:
        ok.append(mx == [1.5 + world - 1, 0.0] and sm == [sum(1.5 + r for r in range(world)), 10.0 * world])
        ok.append(bench.reduce_over_ranks([3.0], None, "cpu") == [3.0])
        with open(result_path, "w") as f:
            f.write(" ".join("1" if x else "0" for x in ok))
    dist.destroy_process_group()


def test_rank_shares_cover_the_workload_and_reductions(tmp_path):
    out = str(tmp_path / "res.txt")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    with open(out) as f:
        res = f.read().split()
    assert res == ["1"] * 5, res
