"""Interpolation from images at successive powers (Sect. 1) on the GPU.

poly_eval_vandermonde_solve recovers each (x1, x2) coefficient's terms from
its images and monomial values.  Its result is unique (distinct nonzero nodes
make the transposed Vandermonde matrix invertible), so it is checked bit for
bit against the oracle's Gaussian elimination, against coefficients chosen
beforehand (images made by the oracle's power sums), and end to end against
the input polynomial after a GPU evaluation.
"""
import random

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pe = pytest.importorskip("paper_2004_11571_gb300")

P62 = wl.random_prime(62, 91)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint64)


def _columns(p, sizes, seed, t0, zero_node=False):
    """Random distinct nodes and coefficients per column, images by the oracle."""
    rnd = random.Random(seed)
    off = np.zeros(len(sizes) + 1, np.uint64)
    off[1:] = np.cumsum(sizes)
    rows = max(sizes) if sizes else 0
    z = np.zeros(int(off[-1]), np.uint64)
    c = np.zeros(int(off[-1]), np.uint64)
    img = np.zeros((max(rows, 1), len(sizes)), np.uint64)
    for g, n in enumerate(sizes):
        nodes = set()
        while len(nodes) < n:
            nodes.add(rnd.randrange(1, p))
        nodes = sorted(nodes)
        if zero_node and n:
            nodes[0] = 0
        rnd.shuffle(nodes)
        a, b = int(off[g]), int(off[g + 1])
        z[a:b] = nodes
        c[a:b] = [rnd.randrange(p) for _ in range(n)]
        img[:n, g] = oracle.power_sums(p, z[a:b], c[a:b], t0, n)
    return off, z, c, img


@pytest.mark.parametrize("p", [P62, wl.random_prime(50, 92), 1_000_003])
@pytest.mark.parametrize("t0", [0, 1, 6])
def test_matches_oracle_gauss(p, t0):
    # Tree levels with ragged ends, tiles of 128 and a partial last tile.
    sizes = [1, 2, 3, 5, 0, 8, 31, 64, 127, 128, 129, 7]
    off, z, c, img = _columns(p, sizes, seed=p % 1000 + t0, t0=t0)
    got = _host(pe.vandermonde_solve(p, off, _dev(z), _dev(img), t0=t0))
    assert got.tolist() == c.tolist()
    for g, n in enumerate(sizes):
        a, b = int(off[g]), int(off[g + 1])
        if n <= 64:
            ref = oracle.tvandermonde_solve(p, z[a:b], img[:n, g], t0)
            assert got[a:b].tolist() == ref.tolist()


def test_large_columns_round_trip():
    """Columns of 1,000 to 3,000 terms (tree depth 12), images by the oracle's
    power sums: the unique solution is the coefficients chosen beforehand."""
    p = P62
    sizes = [3000, 1, 1024, 1025, 17]
    off, z, c, img = _columns(p, sizes, seed=5, t0=1)
    got = _host(pe.vandermonde_solve(p, off, _dev(z), _dev(img), t0=1))
    assert got.tolist() == c.tolist()


def test_strided_images_and_extra_rows():
    p = P62
    sizes = [4, 9, 2]
    off, z, c, img = _columns(p, sizes, seed=7, t0=1)
    big = np.zeros((20, 11), np.uint64)
    big[: img.shape[0], 3:3 + len(sizes)] = img
    dev = _dev(big)[:, 3:3 + len(sizes)]            # rows = 20 >= 9, lda = 11
    got = _host(pe.vandermonde_solve(p, off, _dev(z), dev, t0=1))
    assert got.tolist() == c.tolist()


def test_zero_node_and_singular_columns():
    p = P62
    off, z, c, img = _columns(p, [3, 4], seed=9, t0=0, zero_node=True)
    got = _host(pe.vandermonde_solve(p, off, _dev(z), _dev(img), t0=0))
    assert got.tolist() == c.tolist()                 # a zero node is fine at t0 = 0
    off1, z1, _, img1 = _columns(p, [3, 4], seed=9, t0=1, zero_node=True)
    with pytest.raises(pe.PolyEvalError) as e:
        pe.vandermonde_solve(p, off1, _dev(z1), _dev(img1), t0=1)
    assert e.value.status == pe.PE_ERR_SINGULAR
    zr = z.copy()
    zr[4] = zr[5]                                      # repeated node in column 1
    with pytest.raises(pe.PolyEvalError) as e:
        pe.vandermonde_solve(p, off, _dev(zr), _dev(img), t0=0)
    assert e.value.status == pe.PE_ERR_SINGULAR and "coefficient 1" in str(e.value)
    zb = z.copy()
    zb[2] = p + 1
    with pytest.raises(pe.PolyEvalError) as e:
        pe.vandermonde_solve(p, off, _dev(zb), _dev(img), t0=0)
    assert e.value.status == pe.PE_ERR_NOT_REDUCED


def test_argument_errors():
    p = P62
    off, z, c, img = _columns(p, [5], seed=1, t0=1)
    with pytest.raises(pe.PolyEvalError):
        pe.vandermonde_solve(p, off, _dev(z), _dev(img[:4]), t0=1)      # fewer rows than terms
    with pytest.raises(pe.PolyEvalError):
        pe.vandermonde_solve(p + 1, off, _dev(z), _dev(img), t0=1)      # even modulus
    with pytest.raises(pe.PolyEvalError):
        pe.vandermonde_solve(p, np.array([0, 3, 2], np.uint64), _dev(z), _dev(img), t0=1)
    empty = pe.vandermonde_solve(p, np.zeros(1, np.uint64), _dev(z), _dev(img), t0=1)
    assert empty.numel() == 0


def _monomial_values(w):
    z = np.ones(w.s, dtype=object)
    for j in range(w.n - 2):
        z = [int(zi) * pow(int(w.beta[j]), int(e), w.p) % w.p for zi, e in zip(z, w.exps[:, 2 + j])]
    return np.array(z, dtype=np.uint64)


@pytest.mark.parametrize("t0", [1, 3])
def test_evaluate_then_interpolate(t0):
    """Sect. 1 end to end: images b_t0..b_t0+u-1 from the GPU evaluation, the
    monomial values from Step A, and the solver give back f's coefficients."""
    w = wl.config_interp(seed=21, s=4000, u=300, n=8)
    poly = pe.Poly.from_workload(w)
    images = poly.run(w.beta, w.T, t0=t0)
    z, off = poly.monomials(w.beta)
    assert _host(z).tolist() == _monomial_values(w).tolist()
    _, tg = oracle.group_keys(w.exps)
    assert off.tolist() == [0] + np.cumsum(np.bincount(tg.astype(np.int64))).tolist()
    c = pe.vandermonde_solve(w.p, off, z, images, t0=t0)
    assert _host(c).tolist() == w.coeffs.tolist()
    poly.close()


def test_interp_workload_full_size():
    """The benchmark's interpolation workload (a factor of the m = 14
    symmetric Toeplitz determinant by size: 34,937 terms, largest coefficient
    9,705 terms): evaluation at 9,705 points then interpolation returns f."""
    w = wl.config_interp()
    poly = pe.Poly.from_workload(w)
    images = poly.run(w.beta, w.T, t0=1)
    z, off = poly.monomials(w.beta)
    c = _host(pe.vandermonde_solve(w.p, off, z, images, t0=1))
    assert c.tolist() == w.coeffs.tolist()
    # The images themselves at sampled cells, by the oracle.
    cell = oracle.CellOracle(w)
    rnd = np.random.default_rng(3)
    ts = rnd.integers(0, w.T, 16)
    gs = rnd.integers(0, poly.G, 16)
    img = _host(images)
    assert img[ts, gs].tolist() == cell(ts + 1, gs).tolist()
    poly.close()
