"""The slot sort (canonicalisation method 0) against the CPU oracle,
through the C ABI, on the cases that steer its control flow: one range or
several first-level ranges, leaves packed from many slots, slots of one
repeated key, oversized slots ordered in sub-ranges, the hand-over to the
range sort, and both methods on the same inputs.

Bars as in test_gpu_parity.py: keys and order bit-exact, FP64 coefficients
within 1e-12 * sum |contribution|, FP32-product modes within 8 * 2^-24 *
sum |contribution|.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 8 * 2.0 ** -24


SLOT, RANGE = 0, 1  # canonicalisation methods; the range sort is the default


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2605_25974_gb300 import paulib
    from paper_2605_25974_gb300.build import build
    build()
    torch.cuda.init()
    yield paulib
    paulib.set_slot_tuning(0, RANGE, 0, 0, 0)


@pytest.fixture(autouse=True)
def default_tuning(lib):
    # every test here runs the slot sort unless it says otherwise
    lib.set_slot_tuning(0, SLOT, 0, 0, 0)
    yield
    lib.set_slot_tuning(0, RANGE, 0, 0, 0)


def check(gx, gz, gc, ox, oz, oc, oabs, tol=TOL64):
    assert gx.shape == ox.shape, (gx.shape, ox.shape)
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz)
    err = np.maximum(np.abs(gc.real - oc.real), np.abs(gc.imag - oc.imag))
    bad = err > tol * oabs
    assert not bad.any(), "max rel err %.3g at %d terms" % (float(np.max(err / oabs)), int(bad.sum()))


def product(lib, a, b, precision="fp64", same=False):
    with lib.PauliSum.from_arrays(a) as ga:
        if same:
            with lib.multiply(ga, ga, precision) as gc:
                out = gc.export()[:3]
        else:
            with lib.PauliSum.from_arrays(b) as gb, lib.multiply(ga, gb, precision) as gc:
                out = gc.export()[:3]
    return out + (lib.last_canon_method(),)


def random_sum(n, m, seed, wmax=24):
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(seed)
    x, z = wl.weighted_random(rng, n, m, 1, min(n, wmax))
    return wl.SumArrays(n, x, z, wl.coeffs_loguniform(rng, m))


@pytest.mark.parametrize("n,ma,mb", [(20, 64, 64), (64, 700, 300), (100, 900, 800), (128, 1500, 1100),
                                     (200, 1200, 1300), (300, 600, 777), (500, 2000, 97), (1024, 333, 101)])
def test_slot_sort_every_key_width(lib, oracle, n, ma, mb):
    # one range (small products) up to several first-level ranges
    # (|A||B| above 1024 x the slot target), ragged sizes, 1..16 words per half
    a = random_sum(n, ma, 10 * n + 1)
    b = random_sum(n, mb, 10 * n + 2)
    x, z, c, meth = product(lib, a, b)
    assert meth == (0, 0)
    check(x, z, c, *oracle.multiply_canonical(n, a.as_tuple(), b.as_tuple())[:4])


@pytest.mark.parametrize("n,m", [(100, 1500), (200, 1100)])
def test_slot_sort_jw_hh_with_heavy_identity(lib, oracle, n, m):
    # H*H: the identity string collects m contributions (a slot of one
    # repeated key), most other strings two
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=n, m=m, seed=3000 + n)
    ox, oz, oc, oabs, ocnt = oracle.multiply_canonical(n, h.as_tuple(), h.as_tuple())
    assert ocnt.max() == m
    for prec, tol in (("fp64", TOL64), ("fp32_fp64merge", TOL32), ("fp32_twosum", TOL32)):
        x, z, c, meth = product(lib, h, h, prec)
        assert meth == (0, 0)
        check(x, z, c, ox, oz, oc, oabs, tol)
    x, z, c, meth = product(lib, h, None, "fp64", same=True)
    assert meth == (0, 0)
    check(x, z, c, ox, oz, oc, oabs)


def test_small_leaves_pack_many_slots(lib, oracle):
    # small slots (target 20 terms) packed into leaves of at most 64 terms
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=100, m=700, seed=77)
    lib.set_slot_tuning(0, 0, 64, 20, 8)
    x, z, c, meth = product(lib, h, h)
    assert meth == (0, 0)
    check(x, z, c, *oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())[:4])


@pytest.mark.parametrize("prec", ["fp64", "fp32_twosum"])
def test_oversized_slots_in_sub_ranges_compress(lib, oracle, prec):
    # slots of about 600 terms and leaves of 256: every slot not holding one
    # repeated key is ordered in sub-ranges by the multi-pass leaf.  Half of
    # the terms are the identity (the smallest key, a slot of one repeated
    # key), so every later slot's output stays below its own terms and the
    # slot sort keeps the call.
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(4100)
    n, m = 100, 60000
    ux, uz = wl.weighted_random(rng, n, 4000, 1, 12)
    idx = rng.integers(0, 4000, m // 2)
    x = np.concatenate([np.zeros((ux.shape[0], m // 2), np.uint64), ux[:, idx]], axis=1)
    z = np.concatenate([np.zeros((uz.shape[0], m // 2), np.uint64), uz[:, idx]], axis=1)
    perm = rng.permutation(m)
    s = wl.SumArrays(n, x[:, perm].copy(), z[:, perm].copy(), wl.coeffs_normal(rng, m))
    lib.set_slot_tuning(0, 0, 256, 600, 16)
    with lib.PauliSum.from_arrays(s) as g, lib.compress(g, prec) as gc:
        gx, gz, gcf, _ = gc.export()
    assert lib.last_canon_method() == (0, 0)
    check(gx, gz, gcf, *oracle.compress(n, s.as_tuple())[:4], TOL64 if prec == "fp64" else TOL32)


def test_oversized_slots_in_sub_ranges_product(lib, oracle):
    # A holds 3,000 copies of one string s and B holds s once: s*s = I gives
    # the smallest key 3,000 contributions, and each s*b_j a repeated key
    # too (most of every range); the products of the random parts fill
    # oversized slots.  The slot sort either orders them in sub-ranges or
    # hands the call to the range sort (an oversized slot whose output could
    # reach its own terms, or a sub-range above a leaf); the sum is the same.
    from paper_2605_25974_gb300 import workloads as wl
    n = 200
    rng = wl.rng_for(4200)
    sx, sz = wl.weighted_random(rng, n, 1, 1, 30)
    ra = random_sum(n, 2000, 4201)
    rb = random_sum(n, 300, 4202)
    a = wl.SumArrays(n, np.concatenate([np.repeat(sx, 3000, axis=1), ra.x], axis=1),
                     np.concatenate([np.repeat(sz, 3000, axis=1), ra.z], axis=1),
                     np.concatenate([wl.coeffs_normal(rng, 3000), ra.c]))
    b = wl.SumArrays(n, np.concatenate([sx, rb.x], axis=1), np.concatenate([sz, rb.z], axis=1),
                     np.concatenate([np.array([0.5 + 0.5j]), rb.c]))
    lib.set_slot_tuning(0, 0, 256, 600, 16)
    x, z, c, meth = product(lib, a, b)
    assert meth == (0, 0) or (meth[0] == 1 and meth[1] & ~(64 | 128) == 0), meth
    check(x, z, c, *oracle.multiply_canonical(n, a.as_tuple(), b.as_tuple())[:4])


def test_hand_over_to_range_sort(lib, oracle):
    # distinct products only and oversized slots: the first oversized slot's
    # output would reach its own terms, so the slot sort hands the call to the
    # range sort (bit 64), which gives the same canonical sum
    a = random_sum(150, 800, 91)
    b = random_sum(150, 600, 92)
    lib.set_slot_tuning(0, 0, 64, 2000, 8)
    x, z, c, meth = product(lib, a, b)
    assert meth[0] == 1 and meth[1] & 64
    check(x, z, c, *oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple())[:4])


def test_both_methods_same_keys(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=200, m=900, seed=5)
    ox, oz, oc, oabs, _ = oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())
    for method in (1, 0):
        lib.set_slot_tuning(0, method)
        x, z, c, meth = product(lib, h, h)
        assert meth == (method, 0)
        check(x, z, c, ox, oz, oc, oabs)


def test_compress_through_slot_sort(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(78)
    for n, m, distinct in ((30, 5000, 700), (300, 40000, 900), (64, 3000, 3000)):
        ux, uz = wl.weighted_random(rng, n, distinct, 1, 12)
        idx = rng.integers(0, distinct, m)
        s = wl.SumArrays(n, ux[:, idx].copy(), uz[:, idx].copy(), wl.coeffs_normal(rng, m),
                         rng.integers(0, 4, m).astype(np.uint8))
        with lib.PauliSum.from_arrays(s) as g, lib.compress(g) as gc:
            x, z, c, _ = gc.export()
        assert lib.last_canon_method() == (0, 0)
        check(x, z, c, *oracle.compress(n, s.as_tuple())[:4])


def test_slot_tuning_argument_checks(lib):
    for bad in ((0, 2, -1, -1, -1), (0, -1, 8, -1, -1), (0, -1, 5000, -1, -1), (0, -1, -1, -1, 65),
                (0, -1, -1, -2, -1)):
        with pytest.raises(lib.PaulibError, match="INVALID_ARG"):
            lib.set_slot_tuning(*bad)
