"""Continuous-batching server (GPU): results are bit-exact alone and in a mix
of concurrent requests, with backpressure and eviction under a memory cap."""
import time

import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2004_11571_gb300 as pe  # noqa: E402


def _out(w, G, pinned):
    if pinned:
        return torch.empty((w.T, G), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    return np.zeros((w.T, G), np.uint64)


def _G(w):
    return oracle.group_keys(w.exps)[0].shape[0]


def test_alone_and_in_mix_are_identical():
    pool = wl.config_batched(seed=606, count=16, s_min=300, s_max=40_000)
    srv = pe.Server(streams=3, max_epoch_jobs=8)
    a = pool[0]
    rid = srv.register(a.p, a.coeffs, a.exps)
    out_alone = _out(a, _G(a), True)
    t, _ = srv.submit(a.beta, a.T, out_alone, resident_id=rid)
    assert srv.poll(t) == 0
    _, ref = oracle.eval_direct(a)
    assert np.array_equal(out_alone, ref)
    # The same request inside a burst of uploads and resident reuses.
    reqs = []
    rnd = np.random.default_rng(1)
    for k in range(60):
        w = pool[k % len(pool)]
        if k % 7 == 3:
            reqs.append((a, a.beta, rid, None, _out(a, _G(a), k % 2 == 0)))
        elif k % 3 == 0 and k > 0:
            beta = wl._uniform_mod(rnd, w.p, w.n - 2, lo=2)
            reqs.append((w, beta, None, (w.p, w.coeffs, w.exps), _out(w, _G(w), k % 2 == 0)))
        else:
            reqs.append((w, w.beta, None, (w.p, w.coeffs, w.exps), _out(w, _G(w), k % 2 == 0)))
    tickets = []
    for k, (w, beta, r, poly, out) in enumerate(reqs):
        tickets.append(srv.submit(beta, w.T, out, poly=poly, resident_id=r or 0, borrow=k % 4 == 1)[0])
    for t in tickets:
        assert srv.poll(t) == 0
    for (w, beta, r, poly, out) in reqs:
        if w is a and beta is a.beta:                # the alone request again, resident or re-uploaded
            assert np.array_equal(out, out_alone)
        else:
            wb = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs, exps=w.exps, beta=beta, T=w.T)
            if w.s * w.T < 2_000_000:
                assert np.array_equal(out, oracle.eval_direct(wb)[1])
            else:
                cells = oracle.CellOracle(wb)
                rr = rnd.integers(0, w.T, 10)
                gg = rnd.integers(0, cells.G, 10)
                assert np.array_equal(out[rr, gg], cells(rr + 1, gg))
    st = srv.stats()
    assert st["completed"] == len(reqs) + 1 and st["epochs"] >= 2 and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_resident_reuse_ids_backpressure_and_eviction():
    p = wl.random_prime(62, 5)
    ws = [wl.make_uniform(n=7, s=20_000, p=p, deg12=10, deg_rest=8, T=64, seed=k) for k in range(6)]
    srv = pe.Server(mem_cap_bytes=6 << 20, max_queue=4, streams=1, max_epoch_jobs=2)
    outs, tickets, ids = [], [], []
    for w in ws[:3]:
        o = _out(w, _G(w), False)
        t, nid = srv.submit(w.beta, w.T, o, poly=(w.p, w.coeffs, w.exps))
        tickets.append(t)
        outs.append(o)
    for t in tickets:
        assert srv.poll(t) == 0
    # reuse an uploaded polynomial by the id it was given
    w = ws[0]
    o = _out(w, _G(w), True)
    nb = wl._uniform_mod(np.random.default_rng(3), w.p, w.n - 2, lo=2)
    t, nid = srv.submit(w.beta, w.T, o, poly=(w.p, w.coeffs, w.exps))
    assert srv.poll(t) == 0 and nid > 0
    o2 = _out(w, _G(w), True)
    t2, _ = srv.submit(nb, w.T, o2, resident_id=nid)
    assert srv.poll(t2) == 0
    wb = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs, exps=w.exps, beta=nb, T=w.T)
    assert np.array_equal(o2, oracle.eval_direct(wb)[1])
    # backpressure: while paused, a full backlog refuses with PE_ERR_ADMISSION
    srv.pause(True)
    refused = 0
    pending = []
    for k in range(40):
        w = ws[k % 6]
        try:
            pending.append(srv.submit(w.beta, w.T, _out(w, _G(w), False), poly=(w.p, w.coeffs, w.exps))[0])
        except pe.PolyEvalError as e:
            assert e.status == pe.PE_ERR_ADMISSION
            refused += 1
    assert len(pending) == 4 and refused == 36
    assert srv.poll(pending[0], 0) == pe.PE_PENDING
    srv.pause(False)
    for t in pending:
        assert srv.poll(t) == 0
    for k in range(12):                              # more uploads than the 6 MB cap holds
        w = ws[k % 6]
        t, _ = srv.submit(w.beta, w.T, _out(w, _G(w), False), poly=(w.p, w.coeffs, w.exps))
        assert srv.poll(t) == 0
    st = srv.stats()
    assert st["rejected"] >= refused
    assert st["evictions"] > 0                      # least-recently-used residents make room
    with pytest.raises(pe.PolyEvalError) as e:
        srv.submit(ws[0].beta, 4, np.zeros((4, 10), np.uint64), resident_id=10_000)
    assert e.value.status == 10
    srv.close()
