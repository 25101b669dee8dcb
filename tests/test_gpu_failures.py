"""Failure paths, made on the host or by the library's own bounded checks (no
GPU fault, trap or hang):

* a user allocator callback that returns NULL on the k-th request: the call
  fails with PAULIB_ERR_OOM, frees everything it had taken, and later calls
  work;
* a range-CTA worklist capacity too small for the split: the kernel sets its
  error word and returns, the call fails with PAULIB_ERR_INTERNAL, and the
  next call (capacity restored) is correct;
* warp-leaf key hashes narrowed to a few bits: different keys of a leaf share
  hashes, the leaf takes its whole-key path, and the result still equals the
  oracle's.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2605_25974_gb300 import paulib
    from paper_2605_25974_gb300.build import build
    build()
    torch.cuda.init()
    paulib.load()
    yield paulib
    paulib.set_debug(1, 0)
    paulib.set_debug(2, 0)


def check(x, z, c, ox, oz, oc, oabs):
    assert x.shape == ox.shape and np.array_equal(x, ox) and np.array_equal(z, oz)
    err = np.maximum(np.abs(c.real - oc.real), np.abs(c.imag - oc.imag))
    assert np.all(err <= TOL64 * oabs)


def product(lib, a, b):
    with lib.PauliSum.from_arrays(a) as ga, lib.PauliSum.from_arrays(b) as gb, lib.multiply(ga, gb) as gc:
        return gc.export()[:3]


def test_allocator_returning_null_gives_oom_and_no_leak(lib, oracle):
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    dev = torch.cuda.current_device()
    live = {}
    state = {"calls": 0, "fail_at": None}
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

    def alloc(nbytes, stream, ctx):
        state["calls"] += 1
        if state["fail_at"] is not None and state["calls"] >= state["fail_at"]:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        live[p] = int(nbytes)
        return p

    def free(ptr, stream, ctx):
        assert ptr in live, "freed a pointer the allocator did not hand out"
        del live[ptr]
        torch.cuda.caching_allocator_delete(ptr)

    cb_a, cb_f = ALLOC(alloc), FREE(free)  # kept alive while installed
    c = lib.load()
    assert c.paulib_set_allocator(ctypes.cast(cb_a, ctypes.c_void_p), ctypes.cast(cb_f, ctypes.c_void_p),
                                  None) == 0
    try:
        h = wl.jw(n=100, m=1200, seed=21)  # two first-level ranges and more
        ga = lib.PauliSum.from_arrays(h)
        gb = lib.PauliSum.from_arrays(h)
        held = dict(live)
        base = state["calls"]
        lib.multiply(ga, gb).close()
        torch.cuda.synchronize()
        per_call = state["calls"] - base
        assert per_call >= 4 and live == held
        for k in sorted({1, 2, per_call // 2, per_call - 1, per_call}):
            state["fail_at"] = state["calls"] + k
            with pytest.raises(lib.PaulibError, match="OOM"):
                lib.multiply(ga, gb)
            torch.cuda.synchronize()
            state["fail_at"] = None
            assert live == held, "allocations left behind after a failure at request %d" % k
        with lib.multiply(ga, gb) as gc:
            x, z, cc, _ = gc.export()
        ga.close()
        gb.close()
        torch.cuda.synchronize()
        assert live == {}
    finally:
        assert c.paulib_set_allocator(None, None, None) == 0
    check(x, z, cc, *oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())[:4])


def test_worklist_overflow_is_reported_and_the_next_call_is_correct(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=100, m=1500, seed=22)
    # coarse ranges 8x the default size, so their split queues several
    # children, and a one-entry worklist: the split overflows
    lib.set_tuning(0, 256, 0, 0, 0)
    lib.set_debug(2, 1)
    try:
        with pytest.raises(lib.PaulibError, match="INTERNAL"):
            product(lib, h, h)
    finally:
        lib.set_debug(2, 0)
        lib.set_tuning(0, 32, 0, 0, 0)
    x, z, c = product(lib, h, h)
    check(x, z, c, *oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())[:4])


@pytest.mark.parametrize("bits", [1, 2, 3])
def test_hash_clash_path_of_the_warp_leaves(lib, oracle, bits):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=100, m=500, seed=23)
    rng = wl.rng_for(24)
    a = wl.SumArrays(200, *wl.weighted_random(rng, 200, 700, 1, 20), wl.coeffs_loguniform(rng, 700))
    b = wl.SumArrays(200, *wl.weighted_random(rng, 200, 90, 1, 20), wl.coeffs_loguniform(rng, 90))
    lib.set_debug(1, bits)
    try:
        for x_, y_ in ((h, h), (a, b)):
            x, z, c = product(lib, x_, y_)
            check(x, z, c, *oracle.multiply_canonical(x_.n, x_.as_tuple(), y_.as_tuple())[:4])
    finally:
        lib.set_debug(1, 0)


def test_debug_argument_checks(lib):
    for knob, value in ((0, 1), (5, 1), (1, 65), (1, -1), (2, 5000)):
        with pytest.raises(lib.PaulibError, match="INVALID_ARG"):
            lib.set_debug(knob, value)
