"""Failure paths without a GPU fault, and guard words around outputs.

poly_eval_debug_fail_alloc makes one chosen device allocation of the library
fail as if memory were exhausted (a fake of the failing call, on the host).
Every entry point must then return PE_ERR_NOMEM (or succeed, if it made fewer
allocations) and leave the library and the handles usable: the next call
gives the oracle's images.  Outputs are written exactly where the layout
says: guard words around them stay untouched.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pe = pytest.importorskip("paper_2004_11571_gb300")

PE_ERR_NOMEM = 5
P62 = wl.random_prime(62, 801)
P_NTT = wl.random_ntt_prime(62, 20, 802)


def _failing(call, nth):
    """Runs call() with the nth allocation failing; the status it ends with."""
    pe.debug_fail_alloc(nth)
    try:
        call()
        return 0
    except pe.PolyEvalError as e:
        return e.status
    finally:
        pe.debug_fail_alloc(0)


@pytest.mark.parametrize("shuffle", [False, True])
def test_create_and_run_survive_failed_allocations(shuffle):
    w = wl.make_zipf(n=6, s=40_000, p=P62, deg12=20, deg_rest=6, T=60, seed=3)
    src = wl.shuffled(w, 4) if shuffle else w          # device create path, or the host sort
    _, ref = oracle.eval_direct(w)
    seen_ok = False
    for nth in range(1, 16):
        st = _failing(lambda: pe.Poly(src.p, src.coeffs, src.exps).close(), nth)
        assert st in (0, PE_ERR_NOMEM)
        seen_ok |= st == 0
    assert seen_ok                                      # past its last allocation, create succeeds
    poly = pe.Poly(src.p, src.coeffs, src.exps)
    for nth in range(1, 12):
        st = _failing(lambda: poly.run(src.beta, src.T), nth)
        assert st in (0, PE_ERR_NOMEM)
        assert np.array_equal(pe.to_u64(poly.run(src.beta, src.T)), ref)   # still correct afterwards
    poly.close()


def test_fast_method_solver_and_batch_survive_failed_allocations():
    w = wl.make_zipf(n=6, s=5_000, p=P_NTT, deg12=6, deg_rest=5, T=150, seed=5)
    _, ref = oracle.eval_direct(w)
    poly = pe.Poly.from_workload(w)
    for nth in range(1, 14):
        st = _failing(lambda: poly.run_fast(w.beta, w.T), nth)
        assert st in (0, PE_ERR_NOMEM)
        assert np.array_equal(pe.to_u64(poly.run_fast(w.beta, w.T)), ref)
    wi = wl.config_interp(seed=8, s=3_000, u=300, n=7)     # columns up to 300 terms (the tree path)
    qi = pe.Poly.from_workload(wi)
    images = qi.run(wi.beta, wi.T)
    z, off = qi.monomials(wi.beta)
    for nth in range(1, 10):
        st = _failing(lambda: pe.vandermonde_solve(wi.p, off, z, images), nth)
        assert st in (0, PE_ERR_NOMEM)
    assert pe.to_u64(pe.vandermonde_solve(wi.p, off, z, images)).tolist() == wi.coeffs.tolist()
    qi.close()
    out = torch.empty((w.T, poly.G), dtype=torch.int64, device="cuda")
    for nth in range(1, 8):
        st = _failing(lambda: pe.Batch([(poly, w.beta, w.T, 1, out)]).close(), nth)
        assert st in (0, PE_ERR_NOMEM)
    batch = pe.Batch([(poly, w.beta, w.T, 1, out)])
    batch.launch()
    torch.cuda.synchronize()
    assert np.array_equal(pe.to_u64(out), ref)
    batch.close()
    poly.close()


def _guarded(rows, cols, guard=4096):
    """A flat int64 buffer with guard words on both sides; the view in the middle."""
    buf = torch.full((guard + rows * cols + guard,), 0x5A5A5A5A5A5A5A5A, dtype=torch.int64, device="cuda")
    return buf, buf[guard:guard + rows * cols].view(rows, cols), guard


def _guards_intact(buf, guard):
    h = buf.cpu().numpy()
    return bool(np.all(h[:guard] == 0x5A5A5A5A5A5A5A5A) and np.all(h[-guard:] == 0x5A5A5A5A5A5A5A5A))


def test_outputs_stay_inside_their_layout():
    w = wl.make_zipf(n=6, s=8_000, p=P_NTT, deg12=10, deg_rest=5, T=97, seed=7)
    _, ref = oracle.eval_direct(w)
    poly = pe.Poly.from_workload(w)
    for run in (poly.run, poly.run_fast):
        buf, out, guard = _guarded(w.T, poly.G)
        run(w.beta, w.T, out=out)
        torch.cuda.synchronize()
        assert np.array_equal(pe.to_u64(out), ref) and _guards_intact(buf, guard)
    # interpolation output: columns of the images of a polynomial with distinct monomials
    wi = wl.config_interp(seed=9, s=3_000, u=200, n=7)
    qi = pe.Poly.from_workload(wi)
    images = qi.run(wi.beta, wi.T)
    z, off = qi.monomials(wi.beta)
    buf, c, guard = _guarded(1, wi.s)
    pe.vandermonde_solve(wi.p, off, z, images, out=c.view(-1))
    torch.cuda.synchronize()
    assert pe.to_u64(c.view(-1)).tolist() == wi.coeffs.tolist() and _guards_intact(buf, guard)
    qi.close()
    poly.close()
