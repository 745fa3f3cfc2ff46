"""Extreme values and maximum sizes, bit for bit against the oracle (GPU).

The lazy products keep values below 4p (Barrett) or 2p (Montgomery, the NTTs)
with 4p < 2^64, and the group sums are 96-bit; a wrong bound overflows first
at the largest prime the library takes (just below 2^62) with coefficients
and multipliers at p - 1, or in one group holding most of the terms.  The
other ends: the smallest odd prime, the primes on either side of the 2^30
switch between the 32- and 64-bit products, the largest prime of Algorithm 2
(below 2^50), 64 evaluated variables, exponents of 65535 and the last point
below 2^64.
"""
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


def _prime_below(x, step=1, residue=None):
    """The largest prime below x (with p = 1 mod residue, if given)."""
    q = x - 1
    if residue:
        q -= (q - 1) % residue
        step = residue
    while not wl.is_prime(q):
        q -= step
    return q


def _prime_above(x):
    q = x + 1
    while not wl.is_prime(q):
        q += 1
    return q


P_TOP = _prime_below(1 << 62)                       # 2^62 - 57
P_TOP_NTT = _prime_below(1 << 62, residue=1 << 13)  # NTTs up to 8192 points
P50_TOP = _prime_below(1 << 50)
P30_TOP = _prime_below(1 << 30)
P30_UP = _prime_above(1 << 30)
TOP = (1 << 64) - 1


def _maximal(w, beta_top=True):
    """w with every coefficient p - 1 and the first multipliers p - 1, p - 2."""
    beta = w.beta.copy()
    if beta_top and beta.size:
        beta[0] = w.p - 1
        if beta.size > 1 and w.p > 3:
            beta[1] = w.p - 2
    return dataclasses.replace(w, coeffs=np.full(w.s, w.p - 1, np.uint64), beta=beta)


def _images(w, variant="auto", tiles=None, fast=False, t0=None):
    poly = pe.Poly.from_workload(w, variant=variant)
    if tiles:
        poly.set_tiles(**tiles)
    run = poly.run_fast if fast else poly.run
    out = run(w.beta, w.T, w.t0 if t0 is None else t0)
    torch.cuda.synchronize()
    keys, got = poly.groups(), pe.to_u64(out)
    poly.close()
    return keys, got


def _check(w, variant="auto", tiles=None, fast=False, t0=None):
    keys_ref, ref = oracle.eval_direct(w, t0=t0)
    keys, got = _images(w, variant, tiles, fast, t0)
    assert np.array_equal(keys, keys_ref)
    bad = np.argwhere(got != ref)
    assert bad.size == 0, f"{len(bad)} cells differ, first {bad[:3].tolist()}"


def test_primes_are_what_they_claim():
    assert P_TOP == (1 << 62) - 57
    assert (P_TOP_NTT - 1) % (1 << 13) == 0 and P_TOP_NTT < (1 << 62)
    assert P50_TOP < (1 << 50) < 2 * P50_TOP and P30_TOP < (1 << 30) < P30_UP


@pytest.mark.parametrize("variant,K", [("barrett64", 1), ("barrett64", 16), ("mont64", 4), ("mont64", 16),
                                       ("auto", 0)])
def test_top_prime_with_maximal_values(variant, K):
    w = _maximal(wl.make_zipf(n=6, s=30_000, p=P_TOP, deg12=8, deg_rest=6, T=70, seed=31))
    tiles = dict(K=K, slabs=2, tchunk=32) if K else None
    _check(w, variant, tiles)
    _check(wl.make_zipf(n=6, s=30_000, p=P_TOP, deg12=8, deg_rest=6, T=70, seed=32), variant, tiles)


def test_one_group_holding_every_term():
    # 400,000 terms of coefficient p - 1 in one (x1, x2) cell: sums of 2^80,
    # hundreds of items per T-chunk meeting in the carry slots
    w = _maximal(wl.make_uniform(n=5, s=400_000, p=P_TOP, deg12=0, deg_rest=9, T=64, seed=33))
    _check(w, "barrett64", dict(K=16, slabs=1, tchunk=32))
    _check(w, "mont64", dict(K=1, slabs=4, tchunk=64))
    _check(w)


@pytest.mark.parametrize("p,variant", [(3, "auto"), (3, "fp64"), (P30_TOP, "barrett32"), (P30_TOP, "barrett64"),
                                       (P30_UP, "auto"), ((1 << 31) - 1, "auto"), (P50_TOP, "fp64")])
def test_boundary_primes(p, variant):
    w = wl.make_zipf(n=6, s=12_000, p=p, deg12=6, deg_rest=7, T=45, seed=34)
    _check(_maximal(w), variant)
    _check(w, variant)


def test_most_variables_and_largest_exponents():
    # n = 66: all 64 evaluated variables
    w = wl.make_uniform(n=66, s=3_000, p=P_TOP, deg12=5, deg_rest=4, T=30, seed=35)
    assert w.beta.size == 64
    _check(w)
    # exponents up to 65535 in every variable (u16 rows; nearly every term its own group)
    big = wl.make_uniform(n=7, s=3_000, p=P_TOP, deg12=65535, deg_rest=65535, T=25, seed=36)
    e = big.exps.copy()
    e[:50] = 65535
    _check(dataclasses.replace(big, exps=e))


def test_last_points_below_two_to_the_64():
    w = wl.make_zipf(n=6, s=8_000, p=P_TOP_NTT, deg12=6, deg_rest=5, T=100, seed=37)
    _check(w, t0=TOP - w.T + 1)                       # the last point is 2^64 - 1
    _check(w, fast=True, t0=TOP - w.T + 1)
    poly = pe.Poly.from_workload(w)
    for run in (poly.run, poly.run_fast):
        with pytest.raises(pe.PolyEvalError) as e:
            run(w.beta, w.T, TOP - w.T + 2)           # one point past it
        assert e.value.status == 1 and "2^64" in str(e.value)
    out = torch.empty((w.T, poly.G), dtype=torch.int64, device="cuda")
    with pytest.raises(pe.PolyEvalError):
        pe.Batch([(poly, w.beta, w.T, TOP, out)])
    poly.close()


def test_fast_method_at_the_top_ntt_prime():
    w = _maximal(wl.make_zipf(n=6, s=20_000, p=P_TOP_NTT, deg12=6, deg_rest=6, T=4096, seed=38))
    _check(w, fast=True)
    w2 = wl.make_zipf(n=6, s=20_000, p=P_TOP_NTT, deg12=6, deg_rest=6, T=1000, seed=39)
    _check(w2, fast=True)


def test_batch_of_extreme_primes():
    ws = [_maximal(wl.make_zipf(n=6, s=9_000, p=P_TOP, deg12=5, deg_rest=6, T=90, seed=40)),
          _maximal(wl.make_zipf(n=7, s=5_000, p=P30_TOP, deg12=4, deg_rest=5, T=33, seed=41)),
          _maximal(wl.make_zipf(n=5, s=4_000, p=P50_TOP, deg12=4, deg_rest=5, T=20, seed=42)),
          _maximal(wl.make_uniform(n=5, s=20_000, p=P_TOP, deg12=0, deg_rest=5, T=64, seed=43))]
    polys = [pe.Poly.from_workload(w, variant="fp64" if w.p == P50_TOP else "auto") for w in ws]
    outs = [torch.empty((w.T, q.G), dtype=torch.int64, device="cuda") for w, q in zip(ws, polys)]
    batch = pe.Batch([(q, w.beta, w.T, w.t0, o) for w, q, o in zip(ws, polys, outs)])
    batch.launch()
    torch.cuda.synchronize()
    for w, o in zip(ws, outs):
        assert np.array_equal(pe.to_u64(o), oracle.eval_direct(w)[1])
    batch.close()
    for q in polys:
        q.close()


def test_solver_at_the_top_prime():
    wi = wl.config_interp(seed=44, s=4_000, u=400, n=7)
    wi = dataclasses.replace(wi, p=P_TOP)             # coefficients and beta stay below the larger prime
    poly = pe.Poly.from_workload(wi)
    images = poly.run(wi.beta, wi.T)
    z, off = poly.monomials(wi.beta)
    c = pe.vandermonde_solve(wi.p, off, z, images)
    torch.cuda.synchronize()
    assert pe.to_u64(c).tolist() == wi.coeffs.tolist()
    poly.close()
