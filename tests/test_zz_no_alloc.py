"""paulib_multiply_noalloc: the canonical product for callers that cannot let
a library allocate device memory (their HBM belongs to their own pool or
fixed budget).  It must give the same result as paulib_multiply on the same
inputs, call after call, using only the library's static scratch array; both
are also compared with the CPU oracle (keys and order bit-exact, coefficients
within 1e-12 * sum |contribution|).

This file is collected last on purpose (pytest orders files by name), so a
run that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-12  # the FP64 tolerance of the other parity tests: |dc| <= TOL64 * sum |contribution|


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2605_25974_gb300 import paulib
    from paper_2605_25974_gb300.build import build
    path = build()
    torch.cuda.init()
    paulib.load()
    c = ctypes.CDLL(path)  # the same already-loaded library
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    c.paulib_multiply_noalloc.argtypes = [i32, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, i64, vp, vp]
    c.paulib_multiply_noalloc.restype = i32
    c.paulib_last_error.restype = ctypes.c_char_p
    return c, paulib


def noalloc(c, a, b, expect=0):
    """Calls the entry point through the C ABI on device copies of a and b;
    returns the result, or the status when it is not OK (then it must be
    ``expect``)."""
    import torch
    dev = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).cuda()
    ax, az, acf = dev(a.x.view(np.int64)), dev(a.z.view(np.int64)), dev(a.c.view(np.float64))
    bx, bz, bcf = dev(b.x.view(np.int64)), dev(b.z.view(np.int64)), dev(b.c.view(np.float64))
    cap = max(a.m * b.m, 1)
    W = a.x.shape[0]
    ox = torch.zeros((W, max(cap, 1)), dtype=torch.int64, device="cuda")
    oz = torch.zeros_like(ox)
    oc = torch.zeros((max(cap, 1), 2), dtype=torch.float64, device="cuda")
    on = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    status = c.paulib_multiply_noalloc(a.n, a.m, ax.data_ptr(), az.data_ptr(), acf.data_ptr(), b.m, bx.data_ptr(),
                                       bz.data_ptr(), bcf.data_ptr(), ox.data_ptr(), oz.data_ptr(), oc.data_ptr(),
                                       cap, on.data_ptr(), st)
    if expect:
        assert status == expect, (status, c.paulib_last_error())
        return status
    assert status == 0, c.paulib_last_error()
    u = int(on.item())
    x = ox[:, :u].cpu().numpy().view(np.uint64)
    z = oz[:, :u].cpu().numpy().view(np.uint64)
    cc = oc[:u].cpu().numpy().copy().view(np.complex128).reshape(u)
    return x, z, cc


def with_existing_entry_point(paulib, a, b):
    with paulib.PauliSum.from_arrays(a) as ga, paulib.PauliSum.from_arrays(b) as gb:
        with paulib.multiply(ga, gb, "fp64") as gc:
            x, z, c, _ = gc.export()
    return x, z, c


def check_same(got, ref, oabs):
    x, z, c = got
    rx, rz, rc = ref
    assert x.shape == rx.shape and np.array_equal(x, rx) and np.array_equal(z, rz)
    err = np.maximum(np.abs(c.real - rc.real), np.abs(c.imag - rc.imag))
    assert np.all(err <= TOL64 * oabs)


def test_two_calls_in_a_row_match_the_allocating_entry_point(lib, oracle):
    c, paulib = lib
    from paper_2605_25974_gb300 import workloads as wl
    # first call: a duplicate-heavy H*H near the product limit (255^2 = 65025)
    h = wl.jw(n=100, m=255, seed=12)
    # second call: a different, smaller shape, so stale scratch would show
    rng = wl.rng_for(13)
    ax, az = wl.weighted_random(rng, 200, 900, 1, 24)
    bx, bz = wl.weighted_random(rng, 200, 7, 1, 24)
    a2 = wl.SumArrays(200, ax, az, wl.coeffs_loguniform(rng, 900))
    b2 = wl.SumArrays(200, bx, bz, wl.coeffs_loguniform(rng, 7))
    for a, b in ((h, h), (a2, b2)):
        got = noalloc(c, a, b)
        ref = with_existing_entry_point(paulib, a, b)
        ox, oz, oc, oabs, _ = oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple())
        check_same(got, ref, oabs)
        check_same(got, (ox, oz, oc), oabs)


def test_one_word_keys_and_the_product_limit(lib, oracle):
    # n=20 (one word per half) at 64 x 64, then exactly 256 x 256 = 65536
    # products at n=64, each against the allocating entry point and the oracle
    c, paulib = lib
    from paper_2605_25974_gb300 import workloads as wl
    a, b = wl.tiny()
    rng = wl.rng_for(14)
    a3 = wl.SumArrays(64, *wl.weighted_random(rng, 64, 256, 1, 20), wl.coeffs_normal(rng, 256))
    b3 = wl.SumArrays(64, *wl.weighted_random(rng, 64, 256, 1, 20), wl.coeffs_normal(rng, 256))
    for x, y in ((a, b), (a3, b3)):
        got = noalloc(c, x, y)
        ox, oz, oc, oabs, _ = oracle.multiply_canonical(x.n, x.as_tuple(), y.as_tuple())
        check_same(got, (ox, oz, oc), oabs)
        check_same(got, with_existing_entry_point(paulib, x, y), oabs)


def test_empty_operand_and_tail_bits(lib):
    c, _ = lib
    from paper_2605_25974_gb300 import workloads as wl
    a, b = wl.tiny()
    e = wl.SumArrays(a.n, a.x[:, :0].copy(), a.z[:, :0].copy(), a.c[:0].copy())
    for x, y in ((e, b), (a, e)):
        gx, gz, gc = noalloc(c, x, y)
        assert gx.shape[1] == 0 and gc.shape[0] == 0
    bad = wl.SumArrays(a.n, a.x.copy(), a.z.copy(), a.c.copy())
    bad.x[0, 3] |= np.uint64(1) << np.uint64(30)  # qubit 30 >= n = 20
    assert noalloc(c, bad, b, expect=3) == 3 and b"qubit" in c.paulib_last_error()


def test_sizes_beyond_the_limit_are_rejected(lib):
    c, _ = lib
    out = ctypes.c_int64()
    # 300 x 300 products > 65536: rejected before any device work
    st = c.paulib_multiply_noalloc(20, 300, 1, 1, 1, 300, 1, 1, 1, 1, 1, 1, 90000, ctypes.addressof(out), None)
    assert st == 7 and b"65536" in c.paulib_last_error()
    st = c.paulib_multiply_noalloc(300, 2, 1, 1, 1, 2, 1, 1, 1, 1, 1, 1, 4, ctypes.addressof(out), None)
    assert st == 7 and b"256 qubits" in c.paulib_last_error()
