"""poly_eval_create for terms already in group order runs on the device
(checks, (x1, x2) groups, exponent packing); other inputs take the host path.
Both must give the same polynomial: the same groups and bit-identical images,
which the oracle checks on every cell.  Sizes are above the device path's
threshold of 16,384 terms."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pe = pytest.importorskip("paper_2004_11571_gb300")

P62 = wl.random_prime(62, 501)


def _check(poly, w, keys_ref, ref):
    assert np.array_equal(poly.groups(), keys_ref)
    assert np.array_equal(pe.to_u64(poly.run(w.beta, w.T)), ref)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.uint32])
def test_sorted_host_input_every_exponent_width(dtype):
    w = wl.make_zipf(n=7, s=40_000, p=P62, deg12=20, deg_rest=9, T=24, seed=3)
    keys_ref, ref = oracle.eval_direct(w)
    poly = pe.Poly(w.p, w.coeffs, w.exps.astype(dtype))
    _check(poly, w, keys_ref, ref)
    poly.close()


def test_wide_exponents_and_device_pointers():
    # x3.. exponents above 255 make the packed rows 16-bit.
    w = wl.make_uniform(n=5, s=30_000, p=P62, deg12=6, deg_rest=700, T=12, seed=4)
    keys_ref, ref = oracle.eval_direct(w)
    for exps in (w.exps.astype(np.uint16), w.exps.astype(np.uint32)):
        poly = pe.Poly(w.p, w.coeffs, exps)
        _check(poly, w, keys_ref, ref)
        poly.close()
    coeffs = torch.from_numpy(w.coeffs.view(np.int64).copy()).cuda()
    dexps = torch.from_numpy(w.exps.astype(np.int32)).cuda()
    poly = pe.Poly(w.p, coeffs, dexps)
    _check(poly, w, keys_ref, ref)
    poly.close()


def test_unsorted_input_falls_back_to_the_host_sort():
    w = wl.make_zipf(n=6, s=50_000, p=P62, deg12=25, deg_rest=6, T=16, seed=5)
    keys_ref, ref = oracle.eval_direct(w)
    u = wl.shuffled(w, seed=6)
    poly = pe.Poly(u.p, u.coeffs, u.exps)
    _check(poly, w, keys_ref, ref)
    poly.close()
    coeffs = torch.from_numpy(u.coeffs.view(np.int64).copy()).cuda()
    dexps = torch.from_numpy(u.exps.astype(np.int32)).cuda()
    poly = pe.Poly(u.p, coeffs, dexps)
    _check(poly, w, keys_ref, ref)
    poly.close()


def test_two_variables_and_one_group():
    w = wl.make_uniform(n=2, s=20_000, p=P62, deg12=3, deg_rest=0, T=9, seed=7)
    keys_ref, ref = oracle.eval_direct(w)
    poly = pe.Poly(w.p, w.coeffs, w.exps)
    _check(poly, w, keys_ref, ref)
    poly.close()
    one = wl.make_uniform(n=4, s=20_000, p=P62, deg12=0, deg_rest=5, T=9, seed=8)
    keys_ref, ref = oracle.eval_direct(one)
    poly = pe.Poly(one.p, one.coeffs, one.exps)
    assert poly.G == 1
    _check(poly, one, keys_ref, ref)
    poly.close()


def test_device_path_errors():
    w = wl.make_zipf(n=6, s=20_000, p=P62, deg12=10, deg_rest=5, T=4, seed=9)
    bad = w.coeffs.copy()
    bad[12_345] = w.p + 3
    with pytest.raises(pe.PolyEvalError) as e:
        pe.Poly(w.p, bad, w.exps)
    assert e.value.status == pe.PE_ERR_NOT_REDUCED and "term 12345" in str(e.value)
    with pytest.raises(pe.PolyEvalError) as e:
        pe.Poly(w.p, torch.from_numpy(bad.view(np.int64)).cuda(), torch.from_numpy(w.exps.astype(np.int32)).cuda())
    assert e.value.status == pe.PE_ERR_NOT_REDUCED
    big = w.exps.astype(np.uint32)
    big[777, 3] = 70_000
    with pytest.raises(pe.PolyEvalError) as e:
        pe.Poly(w.p, w.coeffs, big)
    assert "65535" in str(e.value)
    # The same polynomial is still accepted afterwards (nothing left behind).
    keys_ref, ref = oracle.eval_direct(w)
    poly = pe.Poly(w.p, w.coeffs, w.exps)
    _check(poly, w, keys_ref, ref)
    poly.close()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_page_locked_host_input_is_read_directly(dtype):
    # Terms in page-locked host memory are uploaded by the copy engine without
    # a staging copy; the result must be the same polynomial, also for a
    # coefficient that is not reduced (reported, not uploaded silently).
    w = wl.make_zipf(n=7, s=50_000, p=P62, deg12=20, deg_rest=9, T=20, seed=8)
    keys_ref, ref = oracle.eval_direct(w)
    c = torch.from_numpy(w.coeffs.view(np.int64)).pin_memory().numpy().view(np.uint64)
    e = torch.from_numpy(np.ascontiguousarray(w.exps.astype(dtype))).pin_memory().numpy()
    poly = pe.Poly(w.p, c, e, sorted_hint=True)
    _check(poly, w, keys_ref, ref)
    poly.close()
    c[1234] = np.uint64(w.p)
    with pytest.raises(pe.PolyEvalError) as err:
        pe.Poly(w.p, c, e)
    assert err.value.status == pe.PE_ERR_NOT_REDUCED
