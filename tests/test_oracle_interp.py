"""Pins of the oracle's interpolation functions (CPU only).

Sect. 1: with evaluation points at successive powers beta^t, recovering the
coefficients of one (x1, x2) coefficient with n terms from n of its images is
a transposed Vandermonde system: sum_i c_i z_i^(t0+k) = a_k, k < n, where
z_i = M_i(beta).  The oracle solves it by Gaussian elimination; these tests
pin that solver and the power sums to things that do not run through it:
closed forms for n = 1 and n = 2, exhaustive search over a tiny field, exact
Python integers, and the recovery of a polynomial's coefficients from the
images that the evaluation oracle produces.
"""
import itertools
import random

import numpy as np
import pytest

import oracle
import workloads as wl

P62 = wl.random_prime(62, 77)
P50 = wl.random_prime(50, 78)


def _py_power_sums(p, z, c, t0, K):
    return [sum(ci * pow(zi, t0 + k, p) for zi, ci in zip(z, c)) % p for k in range(K)]


def _distinct_nodes(rnd, p, n, lo=1):
    seen = set()
    while len(seen) < n:
        seen.add(rnd.randrange(lo, p))
    return sorted(seen)


@pytest.mark.parametrize("p", [101, P50, P62])
def test_power_sums_match_exact_integers(p):
    rnd = random.Random(p)
    for n in (0, 1, 3, 17):
        z = _distinct_nodes(rnd, p, n)
        c = [rnd.randrange(0, p) for _ in range(n)]
        for t0 in (0, 1, 5):
            got = oracle.power_sums(p, np.array(z, np.uint64), np.array(c, np.uint64), t0, 9)
            assert got.tolist() == _py_power_sums(p, z, c, t0, 9)


@pytest.mark.parametrize("p", [101, P62])
def test_one_term_closed_form(p):
    """n = 1: c = a_0 * z^(-t0)."""
    rnd = random.Random(3)
    for _ in range(20):
        z, a, t0 = rnd.randrange(1, p), rnd.randrange(0, p), rnd.randrange(0, 50)
        c = oracle.tvandermonde_solve(p, np.array([z], np.uint64), np.array([a], np.uint64), t0)
        assert int(c[0]) == a * pow(z, -t0, p) % p


@pytest.mark.parametrize("p", [101, P62])
def test_two_terms_cramer(p):
    """n = 2, Cramer's rule on [[z0^t0, z1^t0], [z0^(t0+1), z1^(t0+1)]]."""
    rnd = random.Random(4)
    for _ in range(20):
        z0, z1 = _distinct_nodes(rnd, p, 2)
        a0, a1 = rnd.randrange(p), rnd.randrange(p)
        t0 = rnd.randrange(0, 6)
        m00, m01, m10, m11 = pow(z0, t0, p), pow(z1, t0, p), pow(z0, t0 + 1, p), pow(z1, t0 + 1, p)
        det = (m00 * m11 - m01 * m10) % p
        inv = pow(det, -1, p)
        c0 = (a0 * m11 - m01 * a1) * inv % p
        c1 = (m00 * a1 - a0 * m10) * inv % p
        c = oracle.tvandermonde_solve(p, np.array([z0, z1], np.uint64), np.array([a0, a1], np.uint64), t0)
        assert c.tolist() == [c0, c1]


def test_exhaustive_search_in_f7():
    """Over F_7, every coefficient vector is the unique preimage of its power sums."""
    p = 7
    for n in (1, 2, 3):
        for z in itertools.combinations(range(1, p), n):
            for t0 in (0, 1, 2):
                images = {}
                for c in itertools.product(range(p), repeat=n):
                    images.setdefault(tuple(_py_power_sums(p, z, c, t0, n)), []).append(c)
                assert len(images) == p ** n                       # the map is a bijection
                for a, (c,) in images.items():
                    got = oracle.tvandermonde_solve(p, np.array(z, np.uint64), np.array(a, np.uint64), t0)
                    assert tuple(got.tolist()) == c


@pytest.mark.parametrize("p,n", [(P62, 40), (P50, 25), (1_000_003, 60)])
def test_round_trip_through_exact_power_sums(p, n):
    rnd = random.Random(n)
    z = _distinct_nodes(rnd, p, n)
    c = [rnd.randrange(0, p) for _ in range(n)]
    for t0 in (0, 1, 7):
        a = _py_power_sums(p, z, c, t0, n)
        got = oracle.tvandermonde_solve(p, np.array(z, np.uint64), np.array(a, np.uint64), t0)
        assert got.tolist() == c


def test_singular_systems_are_reported():
    p = P62
    a = np.arange(1, 4, dtype=np.uint64)
    assert oracle.tvandermonde_solve(p, np.array([5, 9, 5], np.uint64), a, 1) is None   # repeated node
    assert oracle.tvandermonde_solve(p, np.array([0, 9, 4], np.uint64), a, 1) is None   # zero node, t0 > 0
    # With t0 = 0 a zero node is allowed: its column is (1, 0, 0).
    z, c = [0, 9, 4], [11, 22, 33]
    got = oracle.tvandermonde_solve(p, np.array(z, np.uint64),
                                    np.array(_py_power_sums(p, z, c, 0, 3), np.uint64), 0)
    assert got.tolist() == c
    assert oracle.tvandermonde_solve(p, np.zeros(0, np.uint64), np.zeros(0, np.uint64), 1).tolist() == []


def test_interpolation_recovers_polynomial_from_oracle_images():
    """The Sect. 1 use: images b_t of f at beta^t, t = 1..u, and the monomial
    values z_i = M_i(beta) determine every (x1, x2) coefficient of f."""
    w = wl.config_interp(seed=11, s=600, u=40, n=6)
    keys, images = oracle.eval_direct(w)                      # T = u rows, columns by group
    kt = [tuple(k) for k in keys.tolist()]
    col = {k: g for g, k in enumerate(kt)}
    z = [1] * w.s
    for i in range(w.s):
        for j in range(w.n - 2):
            z[i] = z[i] * pow(int(w.beta[j]), int(w.exps[i, 2 + j]), w.p) % w.p
    by_group = {}
    for i in range(w.s):
        by_group.setdefault(col[(int(w.exps[i, 0]), int(w.exps[i, 1]))], []).append(i)
    assert max(len(v) for v in by_group.values()) == w.T
    for g, idx in by_group.items():
        got = oracle.tvandermonde_solve(w.p, np.array([z[i] for i in idx], np.uint64),
                                        images[:len(idx), g], w.t0)
        assert got.tolist() == [int(w.coeffs[i]) for i in idx]


def test_interp_workload_shape():
    w = wl.config_interp(seed=5, s=5000, u=122, n=9)
    assert w.s == 5000 and w.T == 122 and w.t0 == 1
    rows = {tuple(r) for r in w.exps.tolist()}
    assert len(rows) == w.s                                   # distinct monomials
    _, tg = oracle.group_keys(w.exps)
    sizes = np.bincount(tg.astype(np.int64))
    assert sizes.max() == 122 and sizes.min() >= 1
    keys = w.exps[:, 0].astype(np.int64) * (1 << 32) + w.exps[:, 1]
    assert np.all(np.diff(keys) <= 0)                          # sorted by group, descending
