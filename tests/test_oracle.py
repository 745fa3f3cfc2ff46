"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: exact
integer brute force, Fermat's little theorem, ring homomorphisms, the paper's
worked gcd example (Sect. 2.1), Toeplitz determinants (Sect. 2.2.1) and
special cases that reduce to coefficient sums.
"""
import itertools
import os
import random

import numpy as np
import pytest

import oracle
from oracle import brute
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Primes just below powers of two (2^61-1 is a Mersenne prime; the others are
# the largest primes below 2^62, 2^50 and 2^64 listed in published tables).
KNOWN_PRIMES = [2**61 - 1, 2**62 - 57, 2**50 - 27, 101, 65537]
P62 = wl.random_prime(62, 7)
P50 = wl.random_prime(50, 7)


# ------------------------------------------------------------------ F_p ----

@pytest.mark.parametrize("p", KNOWN_PRIMES + [P62, P50])
def test_mulmod_edges_and_fermat(p):
    edges = [0, 1, 2, p - 1, p - 2, (p - 1) // 2] + [1 << k for k in range(0, 62) if (1 << k) < p]
    for a in edges:
        for b in edges:
            assert oracle.mulmod(a, b, p) == (a * b) % p
            assert oracle.addmod(a, b, p) == (a + b) % p
    rnd = random.Random(p)
    for _ in range(200):
        a = rnd.randrange(1, p)
        assert oracle.powmod(a, p - 1, p) == 1                       # Fermat
        assert oracle.mulmod(a, oracle.powmod(a, p - 2, p), p) == 1  # inverse
        e = rnd.randrange(0, 1 << 40)
        assert oracle.powmod(a, e, p) == pow(a, e, p)


def test_miller_rabin_generator():
    for q in KNOWN_PRIMES:
        assert wl.is_prime(q)
    for c in [2**61 + 1, 2**62 - 1, 561, 1105, 3215031751, 2**50 - 1, 1]:
        assert not wl.is_prime(c)
    sympy = pytest.importorskip("sympy")
    rnd = random.Random(3)
    for _ in range(300):
        c = rnd.randrange(2, 1 << 62)
        assert wl.is_prime(c) == bool(sympy.isprime(c))
    for bits in (50, 62):
        p = wl.random_prime(bits, 11)
        assert (1 << (bits - 1)) <= p < (1 << bits) and sympy.isprime(p)


# ---------------------------------------------------- brute force (P0) ----

def _tiny(seed, p, n, s, d12, dr, T):
    return wl.make_uniform(n=n, s=s, p=p, deg12=d12, deg_rest=dr, T=T, seed=seed, sort=False)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("p", [101, 65537, P62, 2**61 - 1])
def test_direct_matches_brute_force(seed, p):
    rnd = random.Random(seed * 7 + p % 1000)
    n = rnd.randint(2, 5)
    w = _tiny(seed, p, n, rnd.randint(1, 40), rnd.randint(0, 3), rnd.randint(0, 4), rnd.randint(1, 8))
    for t0 in (1, 0, 5):
        keys, out = oracle.eval_direct(w, t0=t0)
        bk, rows = brute.eval_exact(p, w.coeffs, w.exps, w.beta, w.T, t0)
        assert [tuple(k) for k in keys.tolist()] == bk
        assert out.tolist() == rows


def test_cells_and_matrix_match_direct():
    for seed, (n, s, d12, dr, T) in enumerate([(6, 500, 8, 5, 19), (9, 800, 5, 20, 33), (3, 50, 2, 3, 7),
                                                (2, 30, 2, 0, 5), (12, 300, 3, 10, 9)]):
        p = P62 if seed % 2 else P50
        w = _tiny(seed, p, n, s, d12, dr, T)
        keys, out = oracle.eval_direct(w, t0=3)
        k2, out2 = oracle.eval_matrix(w, t0=3)
        assert np.array_equal(keys, k2) and np.array_equal(out, out2)
        G = keys.shape[0]
        rnd = np.random.default_rng(seed)
        tt = rnd.integers(0, T, 40)
        gg = rnd.integers(0, G, 40)
        vals = oracle.eval_cells(w, tt + 3, gg)
        assert np.array_equal(vals, out[tt, gg])


# ------------------------------------------------ ring homomorphisms ----

def _concat(a, b):
    return wl.Workload(p=a.p, n=a.n, coeffs=np.concatenate([a.coeffs, b.coeffs]),
                       exps=np.concatenate([a.exps.astype(np.uint32), b.exps.astype(np.uint32)]),
                       beta=a.beta, T=a.T, t0=a.t0)


def _dense(keys, out, D):
    """Bivariate images as dense [T, D, D] arrays of Python ints."""
    T = out.shape[0]
    img = [[[0] * D for _ in range(D)] for _ in range(T)]
    for g, (d, e) in enumerate(keys.tolist()):
        for r in range(T):
            img[r][d][e] = int(out[r, g])
    return img


@pytest.mark.parametrize("seed", range(4))
def test_eval_is_additive_and_multiplicative(seed):
    p = [P62, P50, 101, 2**61 - 1][seed]
    rnd = random.Random(seed)
    n = rnd.randint(3, 6)
    A = _tiny(seed, p, n, rnd.randint(1, 25), 3, 3, 6)
    B = _tiny(seed + 100, p, n, rnd.randint(1, 25), 3, 3, 6)
    B.beta = A.beta
    D = 8
    ka, oa = oracle.eval_direct(A)
    kb, ob = oracle.eval_direct(B)
    ia, ib = _dense(ka, oa, D), _dense(kb, ob, D)
    # A + B: concatenated term lists
    ks, os_ = oracle.eval_direct(_concat(A, B))
    isum = _dense(ks, os_, D)
    for r in range(A.T):
        for d in range(D):
            for e in range(D):
                assert isum[r][d][e] == (ia[r][d][e] + ib[r][d][e]) % p
    # A * B: naive product of the term lists; images multiply as bivariate polynomials
    ce, ee = [], []
    for i in range(A.s):
        for j in range(B.s):
            ce.append(int(A.coeffs[i]) * int(B.coeffs[j]) % p)
            ee.append([int(x) + int(y) for x, y in zip(A.exps[i], B.exps[j])])
    AB = wl.Workload(p=p, n=n, coeffs=np.array(ce, np.uint64), exps=np.array(ee, np.uint32),
                     beta=A.beta, T=A.T, t0=A.t0)
    kp, op = oracle.eval_direct(AB)
    iprod = _dense(kp, op, 2 * D)
    for r in range(A.T):
        conv = [[0] * (2 * D) for _ in range(2 * D)]
        for d1 in range(D):
            for e1 in range(D):
                if ia[r][d1][e1]:
                    for d2 in range(D):
                        for e2 in range(D):
                            conv[d1 + d2][e1 + e2] += ia[r][d1][e1] * ib[r][d2][e2]
        for d in range(2 * D):
            for e in range(2 * D):
                assert iprod[r][d][e] == conv[d][e] % p


# ---------------------------------------------------- special cases ----

def _coeff_sums(w):
    sums = {}
    for c, e in zip(w.coeffs.tolist(), w.exps.tolist()):
        sums[(e[0], e[1])] = (sums.get((e[0], e[1]), 0) + c) % w.p
    return [sums[k] for k in sorted(sums, reverse=True)]


def test_t0_zero_and_beta_one_give_coefficient_sums():
    w = _tiny(5, P62, 7, 400, 4, 6, 4)
    _, out = oracle.eval_direct(w, t0=0)
    assert out[0].tolist() == _coeff_sums(w)          # beta^0 = (1,...,1)
    w1 = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs, exps=w.exps, beta=np.ones(w.n - 2, np.uint64), T=5)
    _, out1 = oracle.eval_direct(w1)
    for r in range(5):
        assert out1[r].tolist() == _coeff_sums(w)
    w2 = wl.Workload(p=w.p, n=2, coeffs=w.coeffs, exps=w.exps[:, :2].copy(), beta=np.zeros(0, np.uint64), T=3)
    _, out2 = oracle.eval_direct(w2)
    for r in range(3):
        assert out2[r].tolist() == _coeff_sums(w2)


def test_single_term_closed_form():
    rnd = random.Random(9)
    for p in (P62, P50, 101):
        n = 7
        e = [rnd.randint(0, 9) for _ in range(n)]
        c = rnd.randrange(1, p)
        beta = [rnd.randrange(2, p) for _ in range(n - 2)]
        w = wl.Workload(p=p, n=n, coeffs=np.array([c], np.uint64), exps=np.array([e], np.uint32),
                        beta=np.array(beta, np.uint64), T=6, t0=2)
        keys, out = oracle.eval_direct(w)
        assert keys.tolist() == [[e[0], e[1]]]
        for r in range(6):
            t = 2 + r
            want = c
            for b, ej in zip(beta, e[2:]):
                want = want * pow(b, t * ej, p) % p
            assert int(out[r, 0]) == want


def _load_gcd_example():
    polys = {}
    with open(os.path.join(GOLDEN, "paper_gcd_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, body = line.split(":", 1)
            terms = [list(map(int, t.split())) for t in body.split(";")]
            polys[name.strip()] = terms
    return polys


def _wl_from_terms(terms, p, beta, T, t0):
    return wl.Workload(p=p, n=4, coeffs=np.array([t[0] % p for t in terms], np.uint64),
                       exps=np.array([t[1:] for t in terms], np.uint32),
                       beta=np.array(beta, np.uint64), T=T, t0=t0)


def test_paper_gcd_example_closed_forms():
    polys = _load_gcd_example()
    p = P62
    b3, b4 = 123456789, 987654321
    T = 6
    kc, oc = oracle.eval_direct(_wl_from_terms(polys["c"], p, [b3, b4], T, 0))
    kd, od = oracle.eval_direct(_wl_from_terms(polys["d"], p, [b3, b4], T, 0))
    assert kc.tolist() == [[1, 1], [0, 0]]
    assert kd.tolist() == [[0, 0]]
    for t in range(T):
        assert int(oc[t, 0]) == 1
        assert int(oc[t, 1]) == pow(b3 * b4, t, p)
        assert int(od[t, 0]) == (pow(b3, t, p) - pow(b4, t, p)) % p
    assert int(od[0, 0]) == 0          # the unlucky point beta^0 = (1, 1)


def _leibniz_det(mat, mul, add, zero, one):
    m = len(mat)
    total = zero
    for perm in itertools.permutations(range(m)):
        sign = 1
        for i in range(m):
            for j in range(i + 1, m):
                if perm[i] > perm[j]:
                    sign = -sign
        prod = one
        for i in range(m):
            prod = mul(prod, mat[i][perm[i]])
        total = add(total, prod if sign > 0 else mul(prod, None))
    return total


@pytest.mark.parametrize("m", [3, 4, 5])
def test_toeplitz_determinant_two_ways(m):
    """det T_m (Sect. 2.2.1, T_ij = x_|i-j|): evaluate the expanded determinant,
    or evaluate the entries and take the determinant over F_p[x0, x1]."""
    p = P50
    # (1) expand det T_m over Z with exponent-vector dict polynomials in x0..x_{m-1}
    def pmul(a, b):
        if b is None:
            return {k: -v for k, v in a.items()}
        r = {}
        for ka, va in a.items():
            for kb, vb in b.items():
                k = tuple(x + y for x, y in zip(ka, kb))
                r[k] = r.get(k, 0) + va * vb
        return r

    def padd(a, b):
        r = dict(a)
        for k, v in b.items():
            r[k] = r.get(k, 0) + v
        return {k: v for k, v in r.items() if v}

    def var(k):
        e = [0] * m
        e[k] = 1
        return {tuple(e): 1}

    mat = [[var(abs(i - j)) for j in range(m)] for i in range(m)]
    det = _leibniz_det(mat, pmul, padd, {}, {tuple([0] * m): 1})
    terms = sorted(det.items())
    rnd = random.Random(m)
    beta = [rnd.randrange(2, p) for _ in range(m - 2)]
    T, t0 = 4, 1
    w = wl.Workload(p=p, n=m, coeffs=np.array([c % p for _, c in terms], np.uint64),
                    exps=np.array([list(e) for e, _ in terms], np.uint32),
                    beta=np.array(beta, np.uint64), T=T, t0=t0)
    keys, out = oracle.eval_direct(w)

    # (2) entries x_k -> beta_k^t for k >= 2, x0, x1 symbolic; determinant over F_p[x0, x1]
    def bmul(a, b):
        if b is None:
            return {k: (-v) % p for k, v in a.items()}
        r = {}
        for (d1, e1), v1 in a.items():
            for (d2, e2), v2 in b.items():
                k = (d1 + d2, e1 + e2)
                r[k] = (r.get(k, 0) + v1 * v2) % p
        return r

    def badd(a, b):
        r = dict(a)
        for k, v in b.items():
            r[k] = (r.get(k, 0) + v) % p
        return r

    for r in range(T):
        t = t0 + r

        def entry(k):
            if k == 0:
                return {(1, 0): 1}
            if k == 1:
                return {(0, 1): 1}
            return {(0, 0): pow(beta[k - 2], t, p)}

        bm = [[entry(abs(i - j)) for j in range(m)] for i in range(m)]
        img = _leibniz_det(bm, bmul, badd, {}, {(0, 0): 1})
        got = {tuple(k): int(out[r, g]) for g, k in enumerate(keys.tolist())}
        for k in set(img) | set(got):
            assert got.get(k, 0) == img.get(k, 0) % p, (m, t, k)
