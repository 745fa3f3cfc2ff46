"""Batched evaluation (one persistent kernel, device work queue, CUDA graph)
is bit-exact against the oracle and against the plain path (GPU)."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2004_11571_gb300 as pe  # noqa: E402


def _mixed(count, seed, s_max=30_000):
    ws = wl.config_batched(seed=seed, count=count, s_min=200, s_max=s_max)
    return ws


def test_batch_matches_oracle_and_plain():
    ws = _mixed(24, 77)
    variants = ["auto", "barrett64", "mont64"]
    polys, outs, jobs = [], [], []
    for k, w in enumerate(ws):
        v = variants[k % 3]
        if k % 4 == 0 and w.p < (1 << 50):
            v = "fp64"
        poly = pe.Poly.from_workload(w, variant=v)
        out = torch.full((w.T, poly.G), -1, dtype=torch.int64, device="cuda")
        t0 = [1, 0, 17, 1 << 33][k % 4]
        polys.append((poly, t0))
        outs.append(out)
        jobs.append((poly, w.beta, w.T, t0, out))
    batch = pe.Batch(jobs)
    for rep in range(2):                      # the graph is re-launchable
        for o in outs:
            o.fill_(-1)
        batch.launch()
        torch.cuda.synchronize()
        for k, w in enumerate(ws):
            poly, t0 = polys[k]
            got = pe.to_u64(outs[k])
            if w.s * w.T <= 3_000_000:
                keys, ref = oracle.eval_direct(w, t0=t0)
                assert np.array_equal(poly.groups(), keys)
                assert np.array_equal(got, ref), f"job {k}"
            else:
                ref = pe.to_u64(poly.run(w.beta, w.T, t0))
                assert np.array_equal(got, ref), f"job {k}"
                cells = oracle.CellOracle(w)
                rnd = np.random.default_rng(k)
                r = rnd.integers(0, w.T, 8)
                g = rnd.integers(0, cells.G, 8)
                assert np.array_equal(got[r, g], cells(r + t0, g))
    # new beta for one job
    w = ws[3]
    nb = wl._uniform_mod(np.random.default_rng(5), w.p, w.n - 2, lo=2)
    batch.set_beta(3, nb)
    batch.launch()
    torch.cuda.synchronize()
    w2 = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs, exps=w.exps, beta=nb, T=w.T, t0=polys[3][1])
    ref = pe.to_u64(polys[3][0].run(nb, w.T, polys[3][1]))
    assert np.array_equal(pe.to_u64(outs[3]), ref)
    batch.close()


def test_batch_with_30_bit_primes():
    p30 = wl.random_prime(30, 91)
    ws = [wl.make_zipf(n=6 + k % 4, s=5_000 + 3_000 * k, p=p30, deg12=10 + k, deg_rest=8, T=60 + 20 * k, seed=k)
          for k in range(6)]
    jobs, outs = [], []
    for k, w in enumerate(ws):
        poly = pe.Poly.from_workload(w, variant="barrett64" if k == 5 else "auto")
        out = torch.full((w.T, poly.G), -1, dtype=torch.int64, device="cuda")
        jobs.append((poly, w.beta, w.T, 2, out))
        outs.append(out)
    batch = pe.Batch(jobs)
    batch.launch()
    torch.cuda.synchronize()
    for w, o in zip(ws, outs):
        _, ref = oracle.eval_direct(w, t0=2)
        assert np.array_equal(pe.to_u64(o), ref)
    batch.close()


def test_batch_edge_jobs():
    p = wl.random_prime(62, 88)
    ws = [wl.make_uniform(n=6, s=1, p=p, deg12=2, deg_rest=3, T=3, seed=1),
          wl.make_uniform(n=2, s=500, p=p, deg12=5, deg_rest=0, T=40, seed=2),
          wl.make_uniform(n=6, s=800, p=p, deg12=0, deg_rest=4, T=1, seed=3),
          wl.make_uniform(n=9, s=7000, p=p, deg12=60, deg_rest=10, T=70, seed=4)]
    jobs, outs = [], []
    for w in ws:
        poly = pe.Poly.from_workload(w)
        out = torch.full((w.T, poly.G), -1, dtype=torch.int64, device="cuda")
        jobs.append((poly, w.beta, w.T, 1, out))
        outs.append(out)
    batch = pe.Batch(jobs)
    batch.launch()
    torch.cuda.synchronize()
    for w, o in zip(ws, outs):
        _, ref = oracle.eval_direct(w)
        assert np.array_equal(pe.to_u64(o), ref)
    batch.close()
    assert pe.Batch([]) is not None


def test_tuner_records_and_plain_uses_it(tmp_path):
    w = wl.make_zipf(n=7, s=60_000, p=wl.random_prime(62, 90), deg12=20, deg_rest=9, T=256, seed=9)
    poly = pe.Poly.from_workload(w)
    tiles, ms = pe.tune(poly, w.T)
    assert tiles["K"] in (1, 2, 4, 8, 12, 16) and ms > 0
    path = str(tmp_path / "tune.jsonl")
    pe.tune_save(path)
    pe.tune_load(path)
    assert "key" in open(path).read()
    _, ref = oracle.eval_direct(wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs, exps=w.exps, beta=w.beta, T=8))
    got = pe.to_u64(poly.run(w.beta, 8))
    assert np.array_equal(got, ref)
    got = pe.to_u64(poly.run(w.beta, w.T))
    cells = oracle.CellOracle(w)
    rnd = np.random.default_rng(0)
    r, g = rnd.integers(0, w.T, 16), rnd.integers(0, cells.G, 16)
    assert np.array_equal(got[r, g], cells(r + 1, g))


def test_shared_power_tables_and_splitting_them():
    """Jobs with the same prime and point share one set of power tables (the
    paired evaluations of the gcd use, Sect. 2.2.2), with the table as wide as
    the largest exponent among them; setting a new point for one job gives it
    its own tables again, for a follower and for the leader."""
    p = wl.random_prime(62, 321)
    beta = np.random.default_rng(5).integers(2, p, size=4, dtype=np.uint64)
    ws = [wl.make_uniform(n=6, s=2_000 + 500 * k, p=p, deg12=6, deg_rest=[3, 9, 5][k], T=40, seed=330 + k)
          for k in range(3)]
    for w in ws:
        w.beta = beta.copy()
    polys = [pe.Poly.from_workload(w) for w in ws]
    outs = [torch.empty((w.T, q.G), dtype=torch.int64, device="cuda") for w, q in zip(ws, polys)]
    batch = pe.Batch([(q, w.beta, w.T, 1, o) for q, w, o in zip(polys, ws, outs)])

    def check():
        batch.launch()
        torch.cuda.synchronize()
        for w, o in zip(ws, outs):
            assert np.array_equal(pe.to_u64(o), oracle.eval_direct(w)[1])

    check()                                              # one table set, width of the widest job (9)
    rng = np.random.default_rng(6)
    ws[2].beta = rng.integers(2, p, size=4, dtype=np.uint64)
    batch.set_beta(2, ws[2].beta)                        # a follower leaves
    check()
    ws[0].beta = rng.integers(2, p, size=4, dtype=np.uint64)
    batch.set_beta(0, ws[0].beta)                        # the leader leaves; job 1 leads alone
    check()
    batch.close()
    for q in polys:
        q.close()


def test_jobs_that_fill_the_gpu_run_as_plain_runs():
    """A job of at least 2^28 term-points leaves the queue for a plain run
    after the graph; small jobs stay in the queue; both kinds, with new
    points set between launches, match the oracle."""
    big = wl.make_zipf(n=7, s=270_000, p=wl.random_prime(62, 91), deg12=20, deg_rest=8, T=1024, seed=92)
    assert big.s * big.T >= 1 << 28
    big50 = wl.make_zipf(n=6, s=135_000, p=wl.random_prime(50, 93), deg12=12, deg_rest=6, T=2048, seed=94,
                         t0=5)
    ws = [big, big50] + _mixed(6, 95)
    polys = [pe.Poly.from_workload(w, variant="fp64" if k == 1 else "auto") for k, w in enumerate(ws)]
    outs = [torch.full((w.T, q.G), -1, dtype=torch.int64, device="cuda") for w, q in zip(ws, polys)]
    batch = pe.Batch([(q, w.beta, w.T, w.t0, o) for w, q, o in zip(ws, polys, outs)])
    info = batch.launches()
    assert info["plain_jobs"] == 2
    assert info["kernels"] == 2 + 3 + 3                 # power tables + queue; three per plain run
    for rep in range(2):
        if rep == 1:                                    # new points for a plain and a queued job
            for k in (0, 3):
                ws[k] = dataclasses.replace(ws[k], beta=wl._uniform_mod(np.random.default_rng(k), ws[k].p,
                                                                          ws[k].n - 2, lo=2))
                batch.set_beta(k, ws[k].beta)
        for o in outs:
            o.fill_(-1)
        batch.launch()
        torch.cuda.synchronize()
        for k, (w, o) in enumerate(zip(ws, outs)):
            ref = oracle.eval_matrix(w)[1] if k < 2 else oracle.eval_direct(w)[1]
            assert np.array_equal(pe.to_u64(o), ref), f"launch {rep}, job {k}"
    batch.close()
    for q in polys:
        q.close()
