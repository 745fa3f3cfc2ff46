"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle.c (on the CPU), compiles it
and runs the pin checks against it: brute force with exact integers, Fermat's
little theorem, the t0 = 0 coefficient sums and the paper's gcd example.  A
mutant that every pin accepts would mean the pins are too weak.
"""
import random

import numpy as np
import pytest

import oracle
from oracle import brute
import workloads as wl

MUTANTS = {
    "dropped coefficient": ("uint64_t v = coeffs[i] % p;\n            for (uint32_t j = 0; j < E; ++j)\n                v = oracle_mulmod(v, pw",
                            "uint64_t v = 1 % p;\n            for (uint32_t j = 0; j < E; ++j)\n                v = oracle_mulmod(v, pw"),
    "wrong exponent column": ("pw[(size_t)j * (dmax + 1) + exps[i * n + 2 + j]]",
                              "pw[(size_t)j * (dmax + 1) + exps[i * n + 1 + j]]"),
    "off-by-one point": ("uint64_t gam = oracle_powmod(beta[j], t, p);",
                         "uint64_t gam = oracle_powmod(beta[j], t + 1, p);"),
    "addmod boundary": ("return s >= p ? s - p : s;", "return s > p ? s - p : s;"),
    "ascending group order": ("return x < y ? 1 : (x > y ? -1 : 0);", "return x < y ? -1 : (x > y ? 1 : 0);"),
    "transposed power operand": ("= oracle_mulmod(pw[(size_t)j * (dmax + 1) + e - 1], gam, p);",
                                 "= oracle_mulmod(pw[(size_t)j * (dmax + 1) + e - 1], beta[j], p);"),
    "powmod skips the top bit": ("while (e) {", "while (e > 1) {"),
    "wrong beta index": ("oracle_powmod(beta[j], t, p);", "oracle_powmod(beta[E - 1 - j], t, p);"),
}


def _pins_hold(lib) -> bool:
    saved = oracle._lib
    oracle._lib = lib
    try:
        for p in (101, 2**61 - 1):
            rnd = random.Random(p)
            for _ in range(20):
                a = rnd.randrange(1, p)
                if oracle.powmod(a, p - 1, p) != 1:
                    return False
            for seed in range(6):
                r = random.Random(seed)
                n = r.randint(3, 5)
                w = wl.make_uniform(n=n, s=r.randint(2, 30), p=p, deg12=2, deg_rest=3, T=4, seed=seed,
                                    sort=False)
                for t0 in (0, 1):
                    keys, out = oracle.eval_direct(w, t0=t0)
                    bk, rows = brute.eval_exact(p, w.coeffs, w.exps, w.beta, w.T, t0)
                    if [tuple(k) for k in keys.tolist()] != bk or out.tolist() != rows:
                        return False
        return True
    finally:
        oracle._lib = saved


def test_unmutated_oracle_passes_pins():
    assert _pins_hold(oracle._load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) >= 1, name
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "mut.so"))
    assert not _pins_hold(lib), f"pins accepted the planted mistake: {name}"


# Mistakes planted in O2 (the matrix method's recurrence, Sect. 2.3), caught
# by brute force with exact integers at t0 = 1 and 3.
O2_MUTANTS = {
    "O2 start power off by one": ("oracle_powmod(m, t0 - 1, p)", "oracle_powmod(m, t0, p)"),
    "O2 sums before advancing": ("v = oracle_mulmod(v, m, p);\n                sums[r] = oracle_addmod(sums[r], v, p);",
                                 "sums[r] = oracle_addmod(sums[r], v, p);\n                v = oracle_mulmod(v, m, p);"),
    "O2 wrong exponent column": ("tab[j][exps[i * n + 2 + j]]", "tab[j][exps[i * n + 1 + j]]"),
    "O2 drops the coefficient": ("oracle_mulmod(coeffs[i] % p, oracle_powmod(m, t0 - 1, p), p)",
                                 "oracle_powmod(m, t0 - 1, p)"),
}


def _o2_pins_hold(lib) -> bool:
    saved = oracle._lib
    oracle._lib = lib
    try:
        for p in (101, 2**61 - 1):
            for seed in range(6):
                r = random.Random(seed)
                w = wl.make_uniform(n=r.randint(3, 5), s=r.randint(2, 30), p=p, deg12=2, deg_rest=3, T=4,
                                    seed=seed, sort=False)
                for t0 in (1, 3):
                    keys, out = oracle.eval_matrix(w, t0=t0)
                    bk, rows = brute.eval_exact(p, w.coeffs, w.exps, w.beta, w.T, t0)
                    if [tuple(k) for k in keys.tolist()] != bk or out.tolist() != rows:
                        return False
        return True
    finally:
        oracle._lib = saved


def test_unmutated_o2_passes_pins():
    assert _o2_pins_hold(oracle._load())


@pytest.mark.parametrize("name", sorted(O2_MUTANTS))
def test_pins_catch_o2_mutant(name, tmp_path):
    old, new = O2_MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, name
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "mut.so"))
    assert not _o2_pins_hold(lib), f"pins accepted the planted mistake: {name}"


# Mistakes planted in the interpolation functions (Sect. 1), caught by the
# closed forms for one and two terms and round trips through power sums
# computed with exact Python integers.
INTERP_MUTANTS = {
    "solver drops t0": ("A[k * (n + 1) + i] = oracle_powmod(z[i], t0 + k, p);",
                        "A[k * (n + 1) + i] = oracle_powmod(z[i], k, p);"),
    "power sums off by one": ("oracle_powmod(z[i], t0 + k, p), p), p);",
                              "oracle_powmod(z[i], t0 + k + 1, p), p), p);"),
    "elimination adds": ("sub ? p - sub : 0", "sub"),
    "wrong inverse exponent": ("oracle_powmod(A[col * (n + 1) + col], p - 2, p)",
                               "oracle_powmod(A[col * (n + 1) + col], p - 1, p)"),
    "solution from the wrong column": ("c[i] = A[i * (n + 1) + n];", "c[i] = A[i * (n + 1) + n - 1];"),
}


def _interp_pins_hold(lib) -> bool:
    saved = oracle._lib
    oracle._lib = lib
    try:
        for p in (101, 2**61 - 1):
            rnd = random.Random(p)
            for n in (1, 2, 5):
                z = rnd.sample(range(1, min(p, 10**6)), n)
                c = [rnd.randrange(p) for _ in range(n)]
                for t0 in (0, 1, 3):
                    exact = [sum(ci * pow(zi, t0 + k, p) for zi, ci in zip(z, c)) % p for k in range(n)]
                    if oracle.power_sums(p, np.array(z, np.uint64), np.array(c, np.uint64), t0, n).tolist() != exact:
                        return False
                    got = oracle.tvandermonde_solve(p, np.array(z, np.uint64), np.array(exact, np.uint64), t0)
                    if got is None or got.tolist() != c:
                        return False
        return True
    finally:
        oracle._lib = saved


def test_unmutated_oracle_passes_interp_pins():
    assert _interp_pins_hold(oracle._load())


@pytest.mark.parametrize("name", sorted(INTERP_MUTANTS))
def test_interp_pins_catch_mutant(name, tmp_path):
    old, new = INTERP_MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, name
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "mut.so"))
    assert not _interp_pins_hold(lib), f"pins accepted the planted mistake: {name}"
