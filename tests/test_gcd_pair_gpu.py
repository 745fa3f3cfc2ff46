"""The gcd use of the evaluations (paper Sect. 2.1 and 2.2.2): f = g c and
h = g c + g d, with c = x1 x2 + x3 x4 and d = x3 - x4 from the paper's example,
evaluated together in one batch at the same beta (GPU).

The images of the products are the products of the images (evaluation at
beta^t is a ring homomorphism onto F_p[x1, x2]), and at the unlucky point
beta^0 the image of d vanishes, so the images of h and f coincide there.
"""
import os
import random

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2004_11571_gb300 as pe  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_gcd_example.txt")


def _example():
    polys = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            name, body = line.split(":", 1)
            polys[name.strip()] = [tuple(map(int, t.split())) for t in body.split(";")]
    return polys


def _mul(a, b, p):
    return [((ca * cb) % p, *[x + y for x, y in zip(ea, eb)]) for ca, *ea in a for cb, *eb in b]


def _workload(terms, p, beta, T):
    return wl.Workload(p=p, n=4, coeffs=np.array([t[0] % p for t in terms], np.uint64),
                       exps=np.array([t[1:] for t in terms], np.uint32), beta=np.array(beta, np.uint64), T=T)


def _image(poly, out, r):
    img = {}
    for g, (d, e) in enumerate(poly.groups().tolist()):
        img[(d, e)] = int(out[r, g])
    return img


def _imul(a, b, p):
    r = {}
    for (d1, e1), x in a.items():
        for (d2, e2), y in b.items():
            r[(d1 + d2, e1 + e2)] = (r.get((d1 + d2, e1 + e2), 0) + x * y) % p
    return {k: v for k, v in r.items() if v}


def _nz(img):
    return {k: v for k, v in img.items() if v}


def test_gcd_pair_in_one_batch():
    ex = _example()
    p = wl.random_prime(62, 404)
    rnd = random.Random(5)
    g = [(rnd.randrange(1, p), rnd.randint(0, 4), rnd.randint(0, 4), rnd.randint(0, 3), rnd.randint(0, 3))
         for _ in range(150)]
    f = _mul(g, ex["c"], p)
    h = f + _mul(g, ex["d"], p)
    beta = [rnd.randrange(2, p), rnd.randrange(2, p)]
    T, t0 = 12, 0
    names = {"g": g, "c": ex["c"], "d": ex["d"], "f": f, "h": h}
    polys, outs, jobs = {}, {}, []
    for name, terms in names.items():
        w = _workload(terms, p, beta, T)
        polys[name] = pe.Poly.from_workload(w)
        outs[name] = torch.full((T, polys[name].G), -1, dtype=torch.int64, device="cuda")
        jobs.append((polys[name], w.beta, T, t0, outs[name]))
    batch = pe.Batch(jobs)
    batch.launch()
    torch.cuda.synchronize()
    res = {k: pe.to_u64(v) for k, v in outs.items()}
    for r in range(T):
        ig, ic, idd = (_image(polys[k], res[k], r) for k in ("g", "c", "d"))
        i_f, i_h = _image(polys["f"], res["f"], r), _image(polys["h"], res["h"], r)
        assert _nz(i_f) == _imul(ig, ic, p)
        cd = {k: (ic.get(k, 0) + idd.get(k, 0)) % p for k in set(ic) | set(idd)}
        assert _nz(i_h) == _imul(ig, cd, p)
        if r + t0 == 0:
            assert not _nz(idd)                      # d(x1, x2, 1, 1) = 0: the unlucky point
            assert _nz(i_h) == _nz(i_f)
        else:
            assert _nz(idd)
    batch.close()
