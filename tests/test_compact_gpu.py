"""Sparse images (only nonzero coefficients, as Algorithm 1 emits them) are
exactly the nonzero entries of the oracle's dense images (GPU)."""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2004_11571_gb300 as pe  # noqa: E402


def _csr(ref):
    rows, cols = np.nonzero(ref)
    row_ptr = np.zeros(ref.shape[0] + 1, np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int64), ref[rows, cols]


def _cancelling(p, seed):
    """Terms that cancel in some groups: every term of a chosen group appears
    again with coefficient p - c, so that group's coefficient is 0 at every point."""
    w = wl.make_uniform(n=5, s=4_000, p=p, deg12=12, deg_rest=6, T=300, seed=seed)
    d, e = int(w.exps[0, 0]), int(w.exps[0, 1])
    sel = (w.exps[:, 0] == d) | (w.exps[:, 1] % 5 == 0)
    neg = ((p - w.coeffs[sel].astype(object)) % p).astype(np.uint64)
    return wl.sort_by_group(wl.Workload(p=p, n=w.n, coeffs=np.concatenate([w.coeffs, neg]),
                                        exps=np.concatenate([w.exps, w.exps[sel]]), beta=w.beta, T=w.T))


@pytest.mark.parametrize("case", ["dense", "cancelling", "t0_zero", "small_prime"])
def test_compact_matches_nonzeros(case):
    p62 = wl.random_prime(62, 71)
    if case == "dense":
        w, t0 = wl.make_zipf(n=7, s=30_000, p=p62, deg12=20, deg_rest=9, T=70, seed=72), 1
    elif case == "cancelling":
        w, t0 = _cancelling(p62, 73), 1
    elif case == "t0_zero":
        # d = x3 - x4 (the paper's unlucky example, Sect. 2.1) vanishes at beta^0
        w = wl.Workload(p=p62, n=4, coeffs=np.array([1, p62 - 1], np.uint64),
                        exps=np.array([[0, 0, 1, 0], [0, 0, 0, 1]], np.uint32),
                        beta=np.array([5, 7], np.uint64), T=6)
        t0 = 0
    else:
        w, t0 = wl.make_uniform(n=6, s=5_000, p=7, deg12=9, deg_rest=5, T=200, seed=74), 1
    keys, ref = oracle.eval_direct(w, t0=t0)
    poly = pe.Poly.from_workload(w)
    dense = poly.run(w.beta, w.T, t0)
    row_ptr, cols, vals = pe.compact(dense)
    torch.cuda.synchronize()
    r_ref, c_ref, v_ref = _csr(ref)
    assert np.array_equal(row_ptr.cpu().numpy(), r_ref)
    assert np.array_equal(cols.cpu().numpy().astype(np.int64), c_ref)
    assert np.array_equal(pe.to_u64(vals), v_ref)
    if case in ("cancelling", "t0_zero", "small_prime"):
        assert r_ref[-1] < ref.size            # some coefficients really are zero
    poly.close()


def test_compact_capacity_and_empty():
    dense = torch.zeros((5, 7), dtype=torch.int64, device="cuda")
    dense[1, 3] = 9
    dense[4, 0] = 2
    row_ptr, cols, vals = pe.compact(dense)
    assert row_ptr.cpu().tolist() == [0, 0, 1, 1, 1, 2]
    assert cols.cpu().tolist() == [3, 0] and vals.cpu().tolist() == [9, 2]
    import ctypes
    nnz = ctypes.c_uint64()
    rp = torch.empty(6, dtype=torch.int64, device="cuda")
    st = pe.lib().poly_eval_compact(dense.data_ptr(), 5, 7, rp.data_ptr(), None, None, 1, ctypes.byref(nnz), None)
    assert st == 1 and nnz.value == 2
    empty = torch.zeros((3, 0), dtype=torch.int64, device="cuda")
    rp, c, v = pe.compact(empty)
    assert rp.cpu().tolist() == [0, 0, 0, 0]
