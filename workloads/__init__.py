"""Seeded synthetic inputs for partial modular polynomial evaluation.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It holds no arithmetic of the evaluation method itself: it
draws primes, coefficients, exponent vectors, evaluation bases and point
counts, and nothing else.

Problem statement (paper Sect. 2.1 and Eq. 1): a polynomial
``f = sum_i a_i x1^{d_i} x2^{e_i} M_i(x3..xn)`` over F_p is evaluated at the
successive powers ``beta^t`` of a point ``beta`` in F_p^{n-2}.  A workload is
therefore ``(p, n, coeffs[s], exps[s, n], beta[n-2], T, t0)``; exponent column
0 is the x1 exponent d_i, column 1 the x2 exponent e_i.

Prime widths follow the paper's discussion of word-size primes: the
floating-point modular product (Algorithm 2) needs p < 2^50, the 64-bit
integer products take p < 2^62.  Primes are drawn as seeded odd candidates and
accepted by a deterministic Miller-Rabin test (bases 2..37, a published result
that is exact for every n < 3.3e24).
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "Workload", "is_prime", "random_prime", "make_uniform", "make_zipf",
    "config_tiny", "config_large", "config_width", "config_batched",
    "served_requests", "sort_by_group", "shuffled", "config_interp", "interp_group_sizes",
    "random_ntt_prime", "inputs_digest", "images_digest", "served_sample", "served_workload",
]

MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (bases 2..37)."""
    n = int(n)
    if n < 2:
        return False
    for q in MR_BASES:
        if n % q == 0:
            return n == q
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in MR_BASES:
        x = pow(a, d, n)
        if x == 1 or x == n - 1:
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def random_prime(bits: int, seed: int) -> int:
    """A prime p with 2^(bits-1) <= p < 2^bits, from seeded odd candidates."""
    if bits < 3 or bits > 63:
        raise ValueError("bits must be in [3, 63]")
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = 1 << (bits - 1), 1 << bits
    while True:
        c = int(rng.integers(lo, hi, dtype=np.uint64)) | 1
        if c < hi and is_prime(c):
            return c


def random_ntt_prime(bits: int, e: int, seed: int) -> int:
    """A prime p = k * 2^e + 1 with 2^(bits-1) <= p < 2^bits (NTTs of every order
    up to 2^e exist in F_p), from seeded odd multipliers k."""
    if not (e + 2 <= bits <= 63):
        raise ValueError("need e + 2 <= bits <= 63")
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = 1 << (bits - 1 - e), 1 << (bits - e)
    while True:
        k = int(rng.integers(lo, hi, dtype=np.uint64)) | 1
        p = k * (1 << e) + 1
        if p < (1 << bits) and is_prime(p):
            return p


@dataclasses.dataclass
class Workload:
    """One evaluation job: terms of f, the base point beta and the points t0..t0+T-1."""
    p: int
    n: int
    coeffs: np.ndarray      # uint64 [s], each < p
    exps: np.ndarray        # uint8/uint16/uint32 [s, n]; column 0 = x1, column 1 = x2
    beta: np.ndarray        # uint64 [n-2], each in [1, p)
    T: int
    t0: int = 1
    name: str = ""

    @property
    def s(self) -> int:
        return int(self.coeffs.shape[0])

    @property
    def term_points(self) -> int:
        return self.s * int(self.T)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _exp_dtype(maxe: int):
    if maxe <= 0xFF:
        return np.uint8
    if maxe <= 0xFFFF:
        return np.uint16
    return np.uint32


def _uniform_mod(rng, p: int, size, lo: int = 0) -> np.ndarray:
    return rng.integers(lo, p, size=size, dtype=np.uint64)


def sort_by_group(w: Workload) -> Workload:
    """Stable sort of the terms by (d, e) in descending lexicographic order
    (paper Sect. 2.3: input sorted in lex order with x1 > x2 > ...)."""
    key = w.exps[:, 0].astype(np.int64) * (1 << 32) + w.exps[:, 1].astype(np.int64)
    order = np.argsort(-key, kind="stable")
    return dataclasses.replace(w, coeffs=w.coeffs[order].copy(), exps=w.exps[order].copy())


def shuffled(w: Workload, seed: int) -> Workload:
    """The same term list in a seeded random order (tests the unsorted path)."""
    order = _rng(seed).permutation(w.s)
    return dataclasses.replace(w, coeffs=w.coeffs[order].copy(), exps=w.exps[order].copy())


def make_uniform(*, n: int, s: int, p: int, deg12: int, deg_rest: int, T: int,
                 seed: int, t0: int = 1, sort: bool = True, name: str = "") -> Workload:
    """Coefficients uniform in [0,p), x1/x2 exponents uniform in 0..deg12,
    x3..xn exponents uniform in 0..deg_rest, beta uniform in [2,p)."""
    if n < 2:
        raise ValueError("n >= 2")
    rng = _rng(seed)
    coeffs = _uniform_mod(rng, p, s)
    dt = _exp_dtype(max(deg12, deg_rest))
    exps = np.empty((s, n), dtype=dt)
    exps[:, :2] = rng.integers(0, deg12 + 1, size=(s, 2)).astype(dt)
    if n > 2:
        exps[:, 2:] = rng.integers(0, deg_rest + 1, size=(s, n - 2)).astype(dt)
    beta = _uniform_mod(rng, p, n - 2, lo=2) if p > 2 else np.ones(n - 2, np.uint64)
    w = Workload(p=p, n=n, coeffs=coeffs, exps=exps, beta=beta, T=T, t0=t0, name=name)
    return sort_by_group(w) if sort else w


def zipf_group_sizes(total: int, ngroups: int, a: float) -> np.ndarray:
    """Group sizes proportional to rank^-a, rounded by largest remainder to
    exactly `total`, at least 1 per group (rank 1 first)."""
    if total < ngroups:
        raise ValueError("need at least one term per group")
    r = np.arange(1, ngroups + 1, dtype=np.float64)
    x = total * r ** (-a) / np.sum(r ** (-a))
    base = np.maximum(1, np.floor(x)).astype(np.int64)
    deficit = total - int(base.sum())
    if deficit > 0:
        frac = x - np.floor(x)
        idx = np.argsort(-frac, kind="stable")[:deficit]
        base[idx] += 1
    while deficit < 0:  # min-1 bumps overshot: take from the largest groups
        i = int(np.argmax(base))
        take = min(-deficit, int(base[i]) - 1)
        base[i] -= take
        deficit += take
    assert int(base.sum()) == total and base.min() >= 1
    return base


def make_zipf(*, n: int, s: int, p: int, deg12: int, deg_rest: int, T: int,
              seed: int, a: float = 1.1, t0: int = 1, name: str = "") -> Workload:
    """Every (d, e) cell with d, e in 0..deg12 is a nonempty group; group sizes
    follow Zipf(a) over the ranks of a seeded permutation of the cells."""
    rng = _rng(seed)
    side = deg12 + 1
    ncell = side * side
    sizes = zipf_group_sizes(s, ncell, a)
    perm = rng.permutation(ncell)            # rank r -> cell perm[r]
    cell_of_term = np.repeat(perm, sizes)     # grouped by rank
    dt = _exp_dtype(max(deg12, deg_rest))
    exps = np.empty((s, n), dtype=dt)
    exps[:, 0] = (cell_of_term // side).astype(dt)
    exps[:, 1] = (cell_of_term % side).astype(dt)
    if n > 2:
        exps[:, 2:] = rng.integers(0, deg_rest + 1, size=(s, n - 2)).astype(dt)
    coeffs = _uniform_mod(rng, p, s)
    beta = _uniform_mod(rng, p, n - 2, lo=2)
    return sort_by_group(Workload(p=p, n=n, coeffs=coeffs, exps=exps, beta=beta, T=T, t0=t0,
                                  name=name))


# ---------------------------------------------------------------------------
# The five workload shapes (sizes as stated for the benchmark configurations).
# ---------------------------------------------------------------------------
SEED_TINY, SEED_LARGE, SEED_WIDTH, SEED_BATCH, SEED_SERVE = 1001, 2002, 3003, 4004, 5005
SEED_INTERP = 6006


def config_tiny(seed: int = SEED_TINY) -> Workload:
    """n=6, 62-bit p, 2,000 terms, x1,x2 in 0..8 (81 groups w.h.p.), x3..x6 in 0..5, T=64."""
    p = random_prime(62, seed)
    return make_uniform(n=6, s=2000, p=p, deg12=8, deg_rest=5, T=64, seed=seed + 1,
                        name="tiny n=6 s=2000 T=64 p62")


def config_large(seed: int = SEED_LARGE, s: int = 1_000_000, T: int = 1024, bits: int = 62) -> Workload:
    """n=9, 62-bit p (or `bits`), 1e6 terms, 71x71 (x1,x2) cells with Zipf(1.1)
    group sizes, x3..x9 in 0..20, T=1024."""
    p = random_prime(bits, seed if bits == 62 else seed + bits)
    return make_zipf(n=9, s=s, p=p, deg12=70, deg_rest=20, T=T, seed=seed + 1, a=1.1,
                     name=f"large n=9 s={s} G=5041 zipf1.1 T={T} p{bits}")


def config_width(bits: int, seed: int = SEED_WIDTH, s: int = 4_000_000, T: int = 4096,
                 ntt: bool = False) -> Workload:
    """The tiny generator at 4e6 terms and T=4096, with a 50-bit or 62-bit prime
    (with ntt=True a prime p = k * 2^20 + 1, as the fast method needs)."""
    p = random_ntt_prime(bits, 20, seed + bits) if ntt else random_prime(bits, seed + bits)
    return make_uniform(n=6, s=s, p=p, deg12=8, deg_rest=5, T=T, seed=seed + 1,
                        name=f"width n=6 s={s} G=81 T={T} p{bits}{' ntt' if ntt else ''}")


def config_batched(seed: int = SEED_BATCH, count: int = 512, s_min: int = 1_000,
                   s_max: int = 1_000_000) -> List[Workload]:
    """`count` independent polynomials: n uniform in 6..12, s log-uniform in
    [s_min, s_max], x1,x2 degree bound D uniform in 5..60, x3.. exponents in 0..10,
    T from {64,256,1024,2048}, 50-bit and 62-bit primes half and half."""
    rng = _rng(seed)
    primes = {50: random_prime(50, seed + 50), 62: random_prime(62, seed + 62)}
    out = []
    for k in range(count):
        n = int(rng.integers(6, 13))
        s = int(round(math.exp(rng.uniform(math.log(s_min), math.log(s_max)))))
        D = int(rng.integers(5, 61))
        T = int(rng.choice([64, 256, 1024, 2048]))
        bits = 50 if k % 2 == 0 else 62
        out.append(make_uniform(n=n, s=s, p=primes[bits], deg12=D, deg_rest=10, T=T,
                                seed=seed * 1000 + k, name=f"batch[{k}] n={n} s={s} D={D} T={T} p{bits}"))
    return out


def served_requests(seed: int = SEED_SERVE, rate: float = 2000.0, duration: float = 60.0,
                    reuse: float = 0.3, pool: Optional[List[Workload]] = None):
    """A Poisson request stream: (arrival_time_s, pool_index, beta or None).

    `beta is None` means a fresh polynomial upload; otherwise the request
    reuses the resident polynomial `pool_index` at the new base point `beta`."""
    rng = _rng(seed)
    if pool is None:
        pool = config_batched(seed=seed)
    t, reqs, seen = 0.0, [], []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        if seen and rng.uniform() < reuse:
            k = int(seen[int(rng.integers(0, len(seen)))])
            w = pool[k]
            beta = _uniform_mod(rng, w.p, w.n - 2, lo=2)
            reqs.append((t, k, beta))
        else:
            k = int(rng.integers(0, len(pool)))
            seen.append(k)
            reqs.append((t, k, None))
    return reqs


SERVED_SAMPLE_FRACTION = 0.011


def served_sample(count: int, seed: int = SEED_SERVE + 1, frac: float = SERVED_SAMPLE_FRACTION) -> np.ndarray:
    """Indices of a seeded sample (about `frac`, at least 1%) of the first
    `count` requests of a served stream; the same indices for any rate."""
    return np.flatnonzero(_rng(seed).random(count) < frac)


def served_workload(pool: List[Workload], req) -> Workload:
    """The evaluation a request (arrival, pool index, beta or None) asks for."""
    _, k, beta = req
    w = pool[k]
    return w if beta is None else dataclasses.replace(w, beta=np.asarray(beta, dtype=np.uint64))


def interp_group_sizes(s: int, u: int) -> np.ndarray:
    """Sizes of the (x1, x2) coefficients of a polynomial to interpolate: s terms,
    the largest coefficient exactly u terms, ceil(4s/u) coefficients whose sizes
    follow rank^-a with a chosen by bisection as large as the cap u allows."""
    if s <= u:
        return np.array([s], np.int64)
    G = -(-4 * s // u)
    lo, hi = 0.0, 4.0
    for _ in range(50):
        a = 0.5 * (lo + hi)
        if zipf_group_sizes(s, G, a)[0] > u:
            hi = a
        else:
            lo = a
    sizes = zipf_group_sizes(s, G, lo)
    deficit = u - int(sizes[0])
    sizes[0] = u
    i = 1
    while deficit > 0:                       # give the extra terms back, largest groups first
        take = min(deficit, int(sizes[i]) - 1)
        sizes[i] -= take
        deficit -= take
        i += 1
    assert int(sizes.sum()) == s and int(sizes.max()) == u and sizes.min() >= 1
    return sizes


def config_interp(seed: int = SEED_INTERP, s: int = 34_937, u: int = 9_705, n: int = 14,
                  bits: int = 62, deg_rest: int = 10) -> Workload:
    """A polynomial to interpolate from its images (Sect. 1): s distinct terms,
    (x1, x2) coefficients sized by interp_group_sizes (the largest u terms),
    x3..xn exponents uniform in 0..deg_rest, distinct within each coefficient,
    nonzero coefficients, T = u points from t0 = 1.  The defaults are the sizes
    the paper gives for a factor of the m = 14 symmetric Toeplitz determinant
    (34,937 terms, largest coefficient 9,705 terms)."""
    if n < 3:
        raise ValueError("n >= 3")
    rng = _rng(seed)
    p = random_prime(bits, seed + bits)
    sizes = interp_group_sizes(s, u)
    G = sizes.shape[0]
    side = int(math.ceil(math.sqrt(G))) + 1
    cells = rng.permutation(side * side)[:G]
    dt = _exp_dtype(max(side, deg_rest))
    exps = np.empty((s, n), dtype=dt)
    at = 0
    for g in range(G):
        k = int(sizes[g])
        rows: set = set()
        while len(rows) < k:
            for r in rng.integers(0, deg_rest + 1, size=(k - len(rows), n - 2)).tolist():
                rows.add(tuple(r))
        exps[at:at + k, 0] = cells[g] // side
        exps[at:at + k, 1] = cells[g] % side
        exps[at:at + k, 2:] = np.array(sorted(rows), dtype=dt)[rng.permutation(k)]
        at += k
    coeffs = _uniform_mod(rng, p, s, lo=1)
    beta = _uniform_mod(rng, p, n - 2, lo=2)
    return sort_by_group(Workload(p=p, n=n, coeffs=coeffs, exps=exps, beta=beta, T=u, t0=1,
                                  name=f"interp n={n} s={s} G={G} u={u} p{bits}"))


# ---------------------------------------------------------------------------
# Digests: stored expected images of the full-size workloads are SHA-256 sums,
# each tied to the exact inputs that produced it.
# ---------------------------------------------------------------------------
def inputs_digest(w: Workload) -> str:
    """SHA-256 of a workload's inputs (p, n, T, t0, coefficients, exponents as
    uint32, beta), independent of the exponent array's integer width."""
    h = hashlib.sha256()
    h.update(np.array([int(w.p), int(w.n), int(w.T), int(w.t0), w.s], dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(w.coeffs, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(w.exps, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(w.beta, dtype="<u8").tobytes())
    return h.hexdigest()


def images_digest(out) -> str:
    """SHA-256 of a (T, G) image array as little-endian uint64, row-major
    (accepts int64 or uint64 numpy arrays holding the same bits)."""
    a = np.ascontiguousarray(np.asarray(out)).view(np.uint64)
    a = np.ascontiguousarray(a, dtype="<u8")
    h = hashlib.sha256()
    h.update(np.array(a.shape, dtype="<u8").tobytes())
    h.update(a.tobytes())
    return h.hexdigest()
