#!/usr/bin/env python3
"""Writes fullsize_images.json: the oracle's images of every full-size workload,
as SHA-256 digests tied to the digests of their inputs.

Calls only the oracle (``oracle.eval_direct``, O1: the definition of the
images, paper Sect. 2.3 below Eq. 1) through ``oracle.shard``, which splits
the groups of one workload, or the workloads of a batch, over the host's
cores.  Nothing here runs or reads the CUDA library.  The digests stand for
outputs too large to store (the 512-job batch alone has about 4.5 GB of
images); a GPU test compares the digest of its own output with them, and
recomputes with the oracle when the inputs it generated have another digest.

    python tests/golden/make_fullsize_digests.py [--procs N] [--only name,...]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import shard  # noqa: E402

OUT = os.path.join(HERE, "fullsize_images.json")

SINGLE = {
    "large": lambda: wl.config_large(),
    "large30": lambda: wl.config_large(bits=30),
    "width62": lambda: wl.config_width(62),
    "width50": lambda: wl.config_width(50),
    "width62ntt": lambda: wl.config_width(62, ntt=True),
}
SERVED_SPAN = {"rate": 2000.0, "duration": 20.0}


def served_cases():
    pool = wl.config_batched(seed=wl.SEED_SERVE)
    reqs = wl.served_requests(seed=wl.SEED_SERVE, pool=pool, **SERVED_SPAN)
    idx = wl.served_sample(len(reqs))
    return pool, reqs, idx


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=0)
    ap.add_argument("--only", default="")
    args = ap.parse_args()
    only = set(filter(None, args.only.split(",")))
    doc = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            doc = json.load(f)
    doc["about"] = ("SHA-256 digests of the oracle's images (O1, the definition) of the full-size workloads, "
                    "each with the digest of its inputs; written by make_fullsize_digests.py")
    single = doc.setdefault("single", {})
    for name, make in SINGLE.items():
        if only and name not in only:
            continue
        w = make()
        t = time.time()
        keys, out = shard.images(w, args.procs)
        single[name] = {"workload": w.name, "inputs": wl.inputs_digest(w), "T": int(w.T), "G": int(keys.shape[0]),
                        "t0": int(w.t0), "keys": wl.images_digest(keys.astype("<u8")),
                        "images": wl.images_digest(out)}
        print(f"{name}: {w.s * w.T:.3e} term-points in {time.time() - t:.1f} s", flush=True)
        _save(doc)
    if not only or "batched" in only:
        ws = wl.config_batched()
        t = time.time()
        dig = shard.many_images(ws, args.procs, digest_only=True)
        doc["batched"] = {"seed": wl.SEED_BATCH, "count": len(ws),
                          "jobs": [{"workload": w.name, "inputs": wl.inputs_digest(w), "images": d}
                                   for w, d in zip(ws, dig)]}
        print(f"batched: {sum(w.s * w.T for w in ws):.3e} term-points in {time.time() - t:.1f} s", flush=True)
        _save(doc)
    if not only or "served" in only:
        pool, reqs, idx = served_cases()
        ws = [wl.served_workload(pool, reqs[i]) for i in idx]
        t = time.time()
        dig = shard.many_images(ws, args.procs, digest_only=True)
        doc["served"] = {"seed": wl.SEED_SERVE, "requests": len(reqs), "fraction": wl.SERVED_SAMPLE_FRACTION,
                         **SERVED_SPAN,
                         "sample": [{"index": int(i), "pool": int(reqs[i][1]), "inputs": wl.inputs_digest(w),
                                     "images": d} for i, w, d in zip(idx, ws, dig)]}
        print(f"served sample: {len(idx)} of {len(reqs)} requests, {sum(w.s * w.T for w in ws):.3e} term-points "
              f"in {time.time() - t:.1f} s", flush=True)
        _save(doc)


def _save(doc):
    tmp = OUT + ".tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, OUT)


if __name__ == "__main__":
    main()
