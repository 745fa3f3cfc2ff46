"""Host-side logic that needs no GPU: the synthetic workload generators and the
benchmark's operation counts for the fast method and the interpolation solver."""
import numpy as np
import pytest

import bench
import oracle
import workloads as wl


def test_ntt_primes():
    for bits, e, seed in [(62, 20, 1), (50, 16, 2), (40, 13, 3)]:
        p = wl.random_ntt_prime(bits, e, seed)
        assert wl.is_prime(p) and (p - 1) % (1 << e) == 0 and p.bit_length() == bits
        # an element of order 2^e exists: Fermat at a random base, then a primitive root of unity
        q = (p - 1) >> e
        w = next(pow(x, q, p) for x in range(2, 100) if pow(pow(x, q, p), 1 << (e - 1), p) == p - 1)
        assert pow(w, 1 << e, p) == 1 and pow(w, 1 << (e - 1), p) == p - 1
    with pytest.raises(ValueError):
        wl.random_ntt_prime(20, 19, 0)


def test_width_workload_ntt_prime():
    w = wl.config_width(62, ntt=True, s=5_000, T=4096)
    assert (w.p - 1) % (1 << 20) == 0 and w.T == 4096 and w.s == 5_000


@pytest.mark.parametrize("s,u", [(5_000, 122), (34_937, 9_705), (100, 100), (50, 122)])
def test_interp_group_sizes(s, u):
    sizes = wl.interp_group_sizes(s, u)
    assert int(sizes.sum()) == s and sizes.min() >= 1 and int(sizes.max()) == min(s, u)


def _fast_counts_brute(off, T):
    """The fast method's products, counted by walking every NTT butterfly."""
    Tp = 64
    while Tp < T:
        Tp *= 2
    def ntt(N):                       # butterflies of one transform
        c, h = 0, N // 2
        while h >= 1:
            c += N // 2
            h //= 2
        return c
    shoup = mont = 0
    for g in range(len(off) - 1):
        n = int(off[g + 1] - off[g])
        for a in range(0, n, Tp):
            d = min(Tp, n - a)
            L = 32
            while L < d:
                for ps in range(0, d, 2 * L):
                    la = min(L, d - ps)
                    if d - ps - la > 0:
                        shoup += 4 * ntt(2 * L) + 2 * (ntt(2 * L) + 2 * L)   # 4 forward, 2 inverse + scaling
                        mont += 3 * 2 * L
                L *= 2
            k = 1
            while k < Tp:
                shoup += 2 * ntt(2 * k) + (ntt(2 * k) + 2 * k) + ntt(2 * k) + (ntt(2 * k) + 2 * k)
                mont += 2 * 2 * k
                k *= 2
            shoup += 2 * ntt(2 * Tp) + ntt(2 * Tp) + 2 * Tp
            mont += 2 * Tp
    return shoup, mont


@pytest.mark.parametrize("sizes,T", [([5000, 1, 70, 4096], 4096), ([300, 64, 65], 100), ([7], 1)])
def test_fast_counts_match_a_walk(sizes, T):
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    assert bench._fast_counts(off, T) == _fast_counts_brute(off, T)


def test_fast_launch_count():
    off = np.array([0, 5000, 5001], np.uint64)
    # leaves on 4096-term blocks reach merge levels 32..2048 (7) for T = 4096
    assert bench._fast_launches(off, 4096) == 5 + 7
    assert bench._fast_launches(np.array([0, 20], np.uint64), 64) == 5


def test_vdm_counts():
    off = np.array([0, 1, 3, 8], np.uint64)         # columns of 1, 2 and 5 terms
    tree, corr, horner, n2 = bench._vdm_counts(off)
    # tree products: 2 terms -> 1*1; 5 terms -> level 1: 1+1, level 2: 2*2, level 4: 4*1
    assert tree == 1 + (1 + 1 + 4 + 4)
    assert corr == 0 + 1 + 10 and horner == 2 * (1 + 4 + 25) and n2 == 30


def test_traffic_reported_only_for_a_captured_shape():
    assert len(bench.STEPB_TRAFFIC_LARGE) >= 2
    for ref in bench.STEPB_TRAFFIC_LARGE:
        shape = dict(ref["shape"], variant=3, chunks=1)          # extra plan keys do not matter
        assert bench.stepb_traffic("large", "barrett64", shape) == ref["bytes"]
        assert bench.stepb_traffic("large", "barrett64", dict(shape, K=8)) is None
        assert bench.stepb_traffic("large", "mont64", shape) is None
        assert bench.stepb_traffic("width62", "barrett64", shape) is None


def test_cpu_baseline_sample_covers_disjoint_groups():
    w = wl.make_zipf(n=5, s=3_000, p=wl.random_prime(62, 9), deg12=6, deg_rest=4, T=4, seed=9)
    _, tg = oracle.group_keys(w.exps)
    parts = [(tg % 4) == r for r in range(4)]
    assert sum(int(p.sum()) for p in parts) == w.s
    assert not np.any(parts[0] & parts[1])
