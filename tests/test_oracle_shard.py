"""The oracle over several processes gives the single-process oracle's images
(CPU).  Splitting the groups over processes is exact because the image of a
group depends on that group's terms alone (paper Sect. 2.3, below Eq. 1)."""
import numpy as np

import oracle
import workloads as wl
from oracle import shard

P62 = wl.random_prime(62, 21)


def test_group_shards_equal_one_process():
    w = wl.make_zipf(n=7, s=30_000, p=P62, deg12=20, deg_rest=9, T=37, seed=5)
    keys, ref = oracle.eval_direct(w)
    for which in ("direct", "matrix"):
        k2, got = shard.images(w, nproc=3, which=which)
        assert np.array_equal(keys, k2) and np.array_equal(got, ref)


def test_many_workloads_and_digests():
    ws = [wl.make_uniform(n=6, s=800 + 97 * k, p=P62 if k % 2 else wl.random_prime(50, 3), deg12=5, deg_rest=4,
                          T=16 + k, seed=k) for k in range(5)]
    outs = shard.many_images(ws, nproc=2)
    digs = shard.many_images(ws, nproc=2, which="matrix", digest_only=True)
    for w, o, d in zip(ws, outs, digs):
        ref = oracle.eval_direct(w)[1]
        assert np.array_equal(o, ref) and d == wl.images_digest(ref)
    # the digest sees one changed cell, the shape and the input digest every input
    bumped = ref.copy()
    bumped[-1, -1] ^= np.uint64(1)
    assert wl.images_digest(bumped) != wl.images_digest(ref)
    assert wl.images_digest(ref.reshape(1, -1)) != wl.images_digest(ref)
    w2 = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs, exps=w.exps, beta=w.beta, T=w.T, t0=w.t0 + 1)
    assert wl.inputs_digest(w2) != wl.inputs_digest(w)
    assert wl.inputs_digest(wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs, exps=w.exps.astype(np.uint32),
                                        beta=w.beta, T=w.T, t0=w.t0)) == wl.inputs_digest(w)
