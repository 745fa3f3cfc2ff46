"""The allocation-free Step B entry point against the oracle (GPU).

poly_eval_stepb_noalloc serves callers that may not allocate device memory
(code running inside another framework's memory pool, an embedded runtime
without allocator access, a process that must not grow after start-up): it
takes device inputs and output only and keeps its scratch in a fixed device
array shared by every call.  Each case makes two calls in a row through the
C ABI and compares both, cell for cell, with the oracle's images (the
definition of the images, paper Sect. 2.3) and with poly_eval_run.  The
larger cases are sized so that the planner has to put several slabs in a
work unit (chain buffers between slabs, groups crossing slab and unit
boundaries) and, in one of them, to cut T into several chunks.
This file runs last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2004_11571_gb300 as pe  # noqa: E402

P62 = wl.random_prime(62, 31)


def _monomials(w):
    """m_i = prod_j beta_j^e_ij mod p with exact Python integers (test-side input)."""
    p = int(w.p)
    m = np.full(w.s, 1, dtype=object)
    for j, b in enumerate(w.beta):
        col = w.exps[:, 2 + j].astype(np.int64)
        table = np.array([pow(int(b), e, p) for e in range(int(col.max()) + 1)], dtype=object)
        m = m * table[col] % p
    return np.array([int(v) for v in m], dtype=np.uint64)


def _group_offsets(w):
    key = w.exps[:, 0].astype(np.int64) * (1 << 32) + w.exps[:, 1].astype(np.int64)
    starts = np.flatnonzero(np.concatenate([[True], key[1:] != key[:-1]]))
    return np.concatenate([starts, [w.s]]).astype(np.uint32)


def _dev_u64(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _noalloc(w, m, goff, t0):
    G = goff.shape[0] - 1
    out = torch.full((w.T, G), -1, dtype=torch.int64, device="cuda")
    pe.stepb_noalloc(w.p, _dev_u64(w.coeffs), _dev_u64(m), torch.from_numpy(goff.view(np.int32)).cuda(),
                     w.T, t0, out)
    torch.cuda.synchronize()
    return pe.to_u64(out)


CASES = {
    # one slab per unit
    "zipf_s20000_T70": lambda: wl.make_zipf(n=7, s=20_000, p=P62, deg12=14, deg_rest=9, T=70, seed=41),
    "uniform_s9001_T64": lambda: wl.make_uniform(n=6, s=9_001, p=P62, deg12=8, deg_rest=5, T=64, seed=42),
    # 2 x 31,250 x 64 x 16 bytes of carries at one slab per unit exceed the
    # scratch: several slabs per unit, one T-chunk
    "zipf_s1e6_T64": lambda: wl.make_zipf(n=7, s=1_000_000, p=P62, deg12=40, deg_rest=9, T=64, seed=43),
    # several slabs per unit and several T-chunks
    "zipf_s32000_T2048": lambda: wl.make_zipf(n=6, s=32_000, p=P62, deg12=14, deg_rest=7, T=2048, seed=44),
}


@pytest.mark.parametrize("t0", [1, 5])
@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_oracle_on_two_calls_in_a_row(name, t0):
    w = CASES[name]()
    goff = _group_offsets(w)
    shape = pe.stepb_noalloc_shape(w.s, w.T)
    if name in ("zipf_s1e6_T64", "zipf_s32000_T2048"):
        assert shape["kslabs"] > 1, shape            # the multi-slab path runs
    if name == "zipf_s32000_T2048":
        assert shape["tchunks"] > 1, shape
    keys, ref = oracle.eval_direct(w, t0=t0)
    assert keys.shape[0] == goff.shape[0] - 1
    m = _monomials(w)
    poly = pe.Poly.from_workload(w, variant="barrett64")
    run = pe.to_u64(poly.run(w.beta, w.T, t0))
    poly.close()
    for call in range(2):                  # two calls in a row share the scratch
        got = _noalloc(w, m, goff, t0)
        bad = np.argwhere(got != ref)
        assert bad.size == 0, f"call {call}: {len(bad)} cells differ from the oracle, first {bad[:3].tolist()}"
        assert np.array_equal(got, run)


def test_noalloc_rejects_oversize_and_host_pointers():
    p = wl.random_prime(62, 32)
    s, T = 1000, 1 << 21          # 2 x T x 16 bytes of carries alone exceed the 32 MiB scratch
    coeffs = torch.zeros(s, dtype=torch.int64, device="cuda")
    goff = torch.tensor([0, s], dtype=torch.int32, device="cuda")
    out = torch.zeros((T, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(pe.PolyEvalError) as e:
        pe.stepb_noalloc(p, coeffs, coeffs, goff, T, 1, out)
    assert "scratch" in str(e.value)
    with pytest.raises(pe.PolyEvalError):
        pe.stepb_noalloc_shape(s, T)
    host = torch.zeros(8, dtype=torch.int64)
    with pytest.raises(pe.PolyEvalError):
        pe.stepb_noalloc(p, host, host, torch.tensor([0, 8], dtype=torch.int32), 4, 1,
                         torch.zeros((4, 1), dtype=torch.int64))


def test_noalloc_malformed_offsets_stay_in_bounds():
    # Offsets that break the contract (past s, decreasing) give unspecified
    # images; the kernel clamps every span to the units that exist, so the
    # guard words around the output stay intact and the next well-formed call
    # is still exact.
    w = wl.make_zipf(n=6, s=40_000, p=P62, deg12=10, deg_rest=5, T=48, seed=45)
    goff = _group_offsets(w)
    G = goff.shape[0] - 1
    m = _monomials(w)
    guard = 64
    bad_past = goff.copy()
    bad_past[G] = w.s + 5000
    bad_past[G // 2] = w.s + 100
    bad_dec = goff.copy()
    bad_dec[3], bad_dec[4] = bad_dec[4], bad_dec[3] - 1
    for bad in (bad_past, bad_dec):
        buf = torch.full((w.T * G + 2 * guard,), 0x5A5A5A5A5A5A5A5A, dtype=torch.int64, device="cuda")
        out = buf[guard:guard + w.T * G].view(w.T, G)
        pe.stepb_noalloc(w.p, _dev_u64(w.coeffs), _dev_u64(m), torch.from_numpy(bad.view(np.int32)).cuda(),
                         w.T, 1, out)
        torch.cuda.synchronize()
        h = buf.cpu()
        assert bool((h[:guard] == 0x5A5A5A5A5A5A5A5A).all()) and bool((h[-guard:] == 0x5A5A5A5A5A5A5A5A).all())
    _, ref = oracle.eval_direct(w)
    assert np.array_equal(_noalloc(w, m, goff, 1), ref)
