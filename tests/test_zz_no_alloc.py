"""The allocation-free Step B entry point agrees with the regular path (GPU).

poly_eval_stepb_noalloc serves callers that may not allocate device memory
(for example code running inside another framework's memory pool): it takes
device inputs and output only and keeps its scratch in a fixed device array.
This file runs last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2004_11571_gb300 as pe  # noqa: E402


def _monomials(w):
    """m_i = prod_j beta_j^e_ij mod p with Python integers (test-side input)."""
    p = int(w.p)
    beta = [int(b) for b in w.beta]
    E = w.n - 2
    out = np.empty(w.s, np.uint64)
    tables = [[pow(b, e, p) for e in range(int(w.exps[:, 2 + j].max()) + 1)] for j, b in enumerate(beta)]
    ex = w.exps[:, 2:].astype(np.int64)
    for i in range(w.s):
        v = 1
        for j in range(E):
            v = v * tables[j][ex[i, j]] % p
        out[i] = v
    return out


def _group_offsets(w):
    key = w.exps[:, 0].astype(np.int64) * (1 << 32) + w.exps[:, 1].astype(np.int64)
    starts = np.flatnonzero(np.concatenate([[True], key[1:] != key[:-1]]))
    return np.concatenate([starts, [w.s]]).astype(np.uint32)


def _dev_u64(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.parametrize("t0", [1, 5])
def test_noalloc_matches_run_on_two_calls_in_a_row(t0):
    p = wl.random_prime(62, 31)
    cases = [wl.make_zipf(n=7, s=20_000, p=p, deg12=14, deg_rest=9, T=70, seed=41),
             wl.make_uniform(n=6, s=9_001, p=p, deg12=8, deg_rest=5, T=64, seed=42)]
    for w in cases:                      # two calls in a row, sharing the scratch
        poly = pe.Poly.from_workload(w, variant="barrett64")
        ref = pe.to_u64(poly.run(w.beta, w.T, t0))
        goff = _group_offsets(w)
        assert goff.shape[0] - 1 == poly.G
        out = torch.full((w.T, poly.G), -1, dtype=torch.int64, device="cuda")
        pe.stepb_noalloc(w.p, _dev_u64(w.coeffs), _dev_u64(_monomials(w)),
                         torch.from_numpy(goff.view(np.int32)).cuda(), w.T, t0, out)
        torch.cuda.synchronize()
        assert np.array_equal(pe.to_u64(out), ref)
        poly.close()


def test_noalloc_rejects_oversize_and_host_pointers():
    p = wl.random_prime(62, 32)
    s, T = 1000, 1 << 21          # 2 x T x 16 bytes of carries alone exceed the 32 MiB scratch
    coeffs = torch.zeros(s, dtype=torch.int64, device="cuda")
    goff = torch.tensor([0, s], dtype=torch.int32, device="cuda")
    out = torch.zeros((T, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(pe.PolyEvalError) as e:
        pe.stepb_noalloc(p, coeffs, coeffs, goff, T, 1, out)
    assert "scratch" in str(e.value)
    host = torch.zeros(8, dtype=torch.int64)
    with pytest.raises(pe.PolyEvalError):
        pe.stepb_noalloc(p, host, host, torch.tensor([0, 8], dtype=torch.int32), 4, 1,
                         torch.zeros((4, 1), dtype=torch.int64))
