"""One term list evaluated modulo several primes (poly_eval_create_like): the
handles share the device exponents and term order and differ only in their
coefficients and prime.  Each prime's images are compared with the oracle on
every cell, alone and inside one batch."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pe = pytest.importorskip("paper_2004_11571_gb300")

PRIMES = [wl.random_prime(62, 601), wl.random_prime(50, 602), wl.random_prime(30, 603)]


def _integer_coeffs(s, seed):
    return np.random.default_rng(seed).integers(0, 1 << 63, size=s, dtype=np.uint64)


def _mod(w, p, ints, beta_seed):
    rng = np.random.default_rng(beta_seed)
    return wl.Workload(p=p, n=w.n, coeffs=(ints % np.uint64(p)).astype(np.uint64), exps=w.exps,
                       beta=rng.integers(2, p, size=w.n - 2, dtype=np.uint64), T=w.T, t0=w.t0)


@pytest.mark.parametrize("shuffle", [False, True])
def test_each_prime_matches_oracle(shuffle):
    base = wl.make_zipf(n=7, s=30_000, p=PRIMES[0], deg12=20, deg_rest=8, T=20, seed=31)
    if shuffle:
        base = wl.shuffled(base, seed=32)     # layout made by the host sort: the permutation is reused
    ints = _integer_coeffs(base.s, 33)
    ws = [_mod(base, p, ints, 40 + k) for k, p in enumerate(PRIMES)]
    layout = pe.Poly(ws[0].p, ws[0].coeffs, ws[0].exps)
    polys = [layout] + [layout.like(w.p, w.coeffs) for w in ws[1:]]
    for poly, w in zip(polys, ws):
        keys, ref = oracle.eval_direct(w)
        assert np.array_equal(poly.groups(), keys)
        assert np.array_equal(pe.to_u64(poly.run(w.beta, w.T)), ref)
    # One batch over the three primes.
    outs = [torch.empty((w.T, polys[0].G), dtype=torch.int64, device="cuda") for w in ws]
    batch = pe.Batch([(poly, w.beta, w.T, 1, o) for poly, w, o in zip(polys, ws, outs)])
    batch.launch()
    torch.cuda.synchronize()
    for w, o in zip(ws, outs):
        assert np.array_equal(pe.to_u64(o), oracle.eval_direct(w)[1])
    batch.close()
    # The shared exponents outlive the layout handle.
    layout.close()
    for poly, w in zip(polys[1:], ws[1:]):
        assert np.array_equal(pe.to_u64(poly.run(w.beta, w.T)), oracle.eval_direct(w)[1])
        poly.close()


def test_device_coefficients_and_errors():
    base = wl.make_uniform(n=5, s=2_000, p=PRIMES[0], deg12=5, deg_rest=6, T=8, seed=51)
    ints = _integer_coeffs(base.s, 52)
    w0, w1 = _mod(base, PRIMES[0], ints, 53), _mod(base, PRIMES[2], ints, 54)
    layout = pe.Poly(w0.p, w0.coeffs, w0.exps)
    dev = torch.from_numpy(w1.coeffs.view(np.int64).copy()).cuda()
    q = layout.like(w1.p, dev)
    assert np.array_equal(pe.to_u64(q.run(w1.beta, w1.T)), oracle.eval_direct(w1)[1])
    q.close()
    with pytest.raises(pe.PolyEvalError) as e:
        layout.like(PRIMES[2], w0.coeffs)                    # 62-bit residues are not reduced mod a 30-bit p
    assert e.value.status == pe.PE_ERR_NOT_REDUCED
    with pytest.raises(pe.PolyEvalError):
        layout.like(PRIMES[0], w0.coeffs, variant="fp64")    # Algorithm 2 needs p < 2^50
    with pytest.raises(pe.PolyEvalError):
        layout.like(PRIMES[0] + 1, w0.coeffs)                # even modulus
    layout.close()
