"""The asymptotically fast method (Sect. 2.3.1, poly_eval_run_fast) gives the
same images as the definition: bit for bit against the oracle on every cell at
test sizes, and against the matrix method (itself checked against the oracle)
plus sampled oracle cells at larger sizes."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pe = pytest.importorskip("paper_2004_11571_gb300")

P_NTT = wl.random_ntt_prime(62, 20, 701)
P_NTT50 = wl.random_ntt_prime(50, 16, 702)


@pytest.mark.parametrize("T,t0", [(1, 1), (5, 0), (64, 1), (100, 7), (300, 1), (1024, 2)])
def test_matches_oracle_every_cell(T, t0):
    # Group sizes from 1 to ~1,600 terms: blocks of one chunk up to several tree levels.
    w = wl.make_zipf(n=6, s=6_000, p=P_NTT, deg12=8, deg_rest=6, T=T, seed=T + t0, a=1.2)
    keys, ref = oracle.eval_direct(w, T=T, t0=t0)
    poly = pe.Poly.from_workload(w)
    got = pe.to_u64(poly.run_fast(w.beta, T, t0=t0))
    assert np.array_equal(got, ref)
    poly.close()


def test_large_groups_match_matrix_method():
    """Groups of ~25,000 terms (several blocks of 4,096 each, full tree depth),
    T = 4,096, a 50-bit NTT prime: identical to the matrix method everywhere
    and to the oracle on sampled cells."""
    w = wl.make_uniform(n=6, s=200_000, p=P_NTT50, deg12=2, deg_rest=7, T=4096, seed=9)
    poly = pe.Poly.from_workload(w)
    fast = pe.to_u64(poly.run_fast(w.beta, w.T))
    plain = pe.to_u64(poly.run(w.beta, w.T))
    assert np.array_equal(fast, plain)
    rng = np.random.default_rng(1)
    ts, gs = rng.integers(0, w.T, 24), rng.integers(0, poly.G, 24)
    assert fast[ts, gs].tolist() == oracle.CellOracle(w)(ts + 1, gs).tolist()
    poly.close()


def test_host_output_and_repeated_runs():
    w = wl.make_zipf(n=5, s=3_000, p=P_NTT, deg12=6, deg_rest=5, T=200, seed=3)
    _, ref = oracle.eval_direct(w)
    poly = pe.Poly.from_workload(w)
    host = np.zeros((w.T, poly.G), np.uint64)
    poly.run_fast(w.beta, w.T, out=host)
    assert np.array_equal(host, ref)
    # A different T rebuilds the plan; the matrix method in between shares Step A's buffers.
    _, ref2 = oracle.eval_direct(w, T=77, t0=3)
    assert np.array_equal(pe.to_u64(poly.run(w.beta, 77, t0=3)), ref2)
    assert np.array_equal(pe.to_u64(poly.run_fast(w.beta, 77, t0=3)), ref2)
    poly.close()


def test_requirements():
    w = wl.make_uniform(n=4, s=500, p=wl.random_prime(62, 703), deg12=3, deg_rest=3, T=16, seed=4)
    poly = pe.Poly.from_workload(w)
    with pytest.raises(pe.PolyEvalError) as e:            # p - 1 without a large power of two
        poly.run_fast(w.beta, 16)
    assert "divisible" in str(e.value)
    poly.close()
    w = wl.make_uniform(n=4, s=500, p=P_NTT, deg12=3, deg_rest=3, T=16, seed=5)
    poly = pe.Poly.from_workload(w)
    with pytest.raises(pe.PolyEvalError):
        poly.run_fast(w.beta, 8192)                         # T above 4096
    poly.close()


def test_tuner_picks_the_faster_method(tmp_path):
    """On large groups at T = 4,096 the fast method wins by a wide margin; after
    tuning, poly_eval_run dispatches to it and still matches the matrix method."""
    w = wl.make_uniform(n=6, s=200_000, p=P_NTT50, deg12=2, deg_rest=7, T=4096, seed=19)
    poly = pe.Poly.from_workload(w)
    plain = pe.to_u64(poly.run(w.beta, w.T))
    pe.tune(poly, w.T)
    assert poly.plan_info(w.T)["method"] == "fast"
    assert np.array_equal(pe.to_u64(poly.run(w.beta, w.T)), plain)
    path = str(tmp_path / "tune.jsonl")
    pe.tune_save(path)
    assert '"method": 1' in open(path).read()
    poly.set_tiles(K=8)                                    # forced tiles: the matrix method again
    assert poly.plan_info(w.T)["method"] == "matrix"
    assert np.array_equal(pe.to_u64(poly.run(w.beta, w.T)), plain)
    poly.close()


def test_two_variables_one_group_and_shared_layout():
    # n = 2: every monomial value is 1, so each image is the coefficient sums.
    w = wl.make_uniform(n=2, s=3_000, p=P_NTT, deg12=3, deg_rest=0, T=130, seed=23)
    _, ref = oracle.eval_direct(w)
    poly = pe.Poly.from_workload(w)
    assert np.array_equal(pe.to_u64(poly.run_fast(w.beta, w.T)), ref)
    poly.close()
    one = wl.make_uniform(n=5, s=9_000, p=P_NTT, deg12=0, deg_rest=6, T=300, seed=24)
    _, ref = oracle.eval_direct(one)
    poly = pe.Poly.from_workload(one)
    assert poly.G == 1
    assert np.array_equal(pe.to_u64(poly.run_fast(one.beta, one.T)), ref)
    # the same terms modulo another NTT prime, sharing the exponents
    p2 = wl.random_ntt_prime(50, 16, 704)
    c2 = (one.coeffs % np.uint64(p2)).astype(np.uint64)
    w2 = wl.Workload(p=p2, n=one.n, coeffs=c2, exps=one.exps, beta=one.beta % np.uint64(p2 - 2) + np.uint64(1),
                     T=one.T, t0=1)
    q = poly.like(p2, c2)
    assert np.array_equal(pe.to_u64(q.run_fast(w2.beta, w2.T)), oracle.eval_direct(w2)[1])
    q.close()
    poly.close()
