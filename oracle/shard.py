"""The oracle over several host cores (test infrastructure).

Only the tests, the smoke check, the benchmark's CPU-baseline leg and the
script that writes the stored full-size digests may use this module.

The image of group g at point t depends on the terms of group g alone (paper
Sect. 2.3, the definition below Eq. 1), so the columns of the output can be
computed by independent processes: share r evaluates, with the single-threaded
oracle, the sub-polynomial made of the groups g with g mod nshare = r, and
its columns are put back in place.  Independent workloads (the jobs of a
batch, the requests of a stream) run one per process, largest first.  Nothing
here changes the arithmetic: every value is computed by ``oracle.eval_direct``
(O1, the definition) or ``oracle.eval_matrix`` (O2, pinned equal to O1).

Processes are spawned, never forked, so callers that have already used a GPU
can use this module safely.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os
from typing import List, Sequence

import numpy as np


def _fn(which):
    import oracle
    if which == "direct":
        return oracle.eval_direct
    if which == "matrix":
        return oracle.eval_matrix
    raise ValueError(f"unknown oracle {which!r}")


def _subset(w, sel):
    import workloads as wl
    return wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs[sel], exps=w.exps[sel], beta=w.beta, T=w.T, t0=w.t0)


def _share(args):
    w, nshare, r, which = args
    import oracle
    _, tg = oracle.group_keys(w.exps)
    sel = (tg % nshare) == r
    if not sel.any():
        return r, np.zeros((w.T, 0), np.uint64)
    _, out = _fn(which)(_subset(w, sel))
    return r, out


def _whole(args):
    idx, w, which, digest_only = args
    _, out = _fn(which)(w)
    if digest_only:
        import workloads as wl
        return idx, wl.images_digest(out)
    return idx, out


def _pool(nproc):
    # A worker that dies raises BrokenProcessPool in the caller instead of
    # leaving it waiting for a result that never comes.
    return cf.ProcessPoolExecutor(max_workers=nproc, mp_context=mp.get_context("spawn"))


def images(w, nproc: int = 0, which: str = "direct"):
    """(keys, out[T, G]) of one workload, its groups split over nproc processes."""
    import oracle
    oracle.build()
    nproc = nproc or os.cpu_count() or 1
    keys, tg = oracle.group_keys(w.exps)
    G = keys.shape[0]
    out = np.zeros((int(w.T), G), np.uint64)
    if G == 0:
        return keys, out
    nshare = min(nproc, G)
    cols = np.arange(G)
    with _pool(nproc) as pool:
        for fut in cf.as_completed([pool.submit(_share, (w, nshare, r, which)) for r in range(nshare)]):
            r, part = fut.result()
            out[:, cols[cols % nshare == r]] = part
    return keys, out


def many_images(ws: Sequence, nproc: int = 0, which: str = "direct", digest_only: bool = False) -> List:
    """Images (or their digests) of independent workloads, one process per
    workload at a time, the costliest first."""
    import oracle
    oracle.build()
    nproc = nproc or os.cpu_count() or 1
    order = sorted(range(len(ws)), key=lambda i: -ws[i].s * int(ws[i].T) * max(ws[i].n - 1, 1))
    res: List = [None] * len(ws)
    with _pool(nproc) as pool:
        for fut in cf.as_completed([pool.submit(_whole, (i, ws[i], which, digest_only)) for i in order]):
            i, val = fut.result()
            res[i] = val
    return res
