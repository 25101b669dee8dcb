"""The persistent batched kernel against the CPU oracle, problem by problem,
through the C ABI, on inputs that steer its control flow:

* random propagation-shaped batches (problems of up to a leaf's capacity in
  one leaf, larger ones split by sampled splitters) at every key width and
  in every precision mode, next to the general multi-kernel pipeline;
* a small leaf capacity (test knob 4), so that small problems split, and
  keys that vary on a few qubits only, so that children split again;
* problems whose products all share one key (the summed-range paths, at the
  top and below a split);
* keys that agree on the leaf's 64-bit window and differ later (whole-key
  comparisons in shared memory);
* empty operands, a right operand too large for the kernel (the general
  pipeline takes the batch), and graph replay of a plan.

Bars as in test_gpu_parity.py: keys and order bit-exact, FP64 coefficients
within 1e-12 * sum |contribution|, FP32-product modes within 8 * 2^-24 *
sum |contribution|.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 8 * 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2605_25974_gb300 import paulib
    from paper_2605_25974_gb300.build import build
    build()
    torch.cuda.init()
    paulib.load()
    yield paulib
    paulib.set_debug(3, 0)
    paulib.set_debug(4, 0)


@pytest.fixture(autouse=True)
def defaults(lib):
    lib.set_debug(3, 0)
    lib.set_debug(4, 0)
    yield
    lib.set_debug(3, 0)
    lib.set_debug(4, 0)


def check(x, z, c, ox, oz, oc, oabs, tol=TOL64):
    assert x.shape == ox.shape, (x.shape, ox.shape)
    assert np.array_equal(x, ox) and np.array_equal(z, oz)
    err = np.maximum(np.abs(c.real - oc.real), np.abs(c.imag - oc.imag))
    bad = err > tol * oabs
    assert not bad.any(), "max rel err %.3g at %d terms" % (float(np.max(err / oabs)), int(bad.sum()))


def run_batch(lib, probs, precision="fp64"):
    As = [lib.PauliSum.from_arrays(a) for a, _ in probs]
    Bs = [lib.PauliSum.from_arrays(b) for _, b in probs]
    outs = lib.multiply_batched(As, Bs, precision)
    res = [o.export()[:3] for o in outs]
    for s in As + Bs + outs:
        s.close()
    return res


def check_batch(lib, oracle, probs, precision="fp64"):
    tol = TOL64 if precision == "fp64" else TOL32
    for (a, b), (x, z, c) in zip(probs, run_batch(lib, probs, precision)):
        check(x, z, c, *oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple())[:4], tol)


def sums(n, m, rng, wmax=32, lo_q=0, hi_q=None):
    """m random strings of weight <= wmax on qubits lo_q .. hi_q - 1."""
    from paper_2605_25974_gb300 import workloads as wl
    hi_q = n if hi_q is None else hi_q
    span = hi_q - lo_q
    sx, sz = wl.low_weight_terms(rng, span, m, min(wmax, span))
    W = (n + 63) // 64
    x = np.zeros((W, m), np.uint64)
    z = np.zeros((W, m), np.uint64)
    for q in range(span):
        w, bit = divmod(q, 64)
        bx = (sx[w] >> np.uint64(bit)) & np.uint64(1)
        bz = (sz[w] >> np.uint64(bit)) & np.uint64(1)
        tw, tb = divmod(lo_q + q, 64)
        x[tw] |= bx << np.uint64(tb)
        z[tw] |= bz << np.uint64(tb)
    return wl.SumArrays(n, x, z, wl.coeffs_loguniform(rng, m))


@pytest.mark.parametrize("n", [20, 100, 200, 500, 1000])
def test_random_batches_every_key_width(lib, oracle, n):
    from paper_2605_25974_gb300 import workloads as wl
    probs = wl.batch(problems=24, n=n, seed=600 + n, amin=1, amax=6000, wmax=min(32, n))
    check_batch(lib, oracle, probs)


@pytest.mark.parametrize("precision", ["fp32_fp64merge", "fp32_twosum"])
def test_random_batch_mixed_precision(lib, oracle, precision):
    from paper_2605_25974_gb300 import workloads as wl
    probs = wl.batch(problems=16, seed=611, amax=8000)
    check_batch(lib, oracle, probs, precision)


def test_persistent_and_general_pipeline_agree(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    probs = wl.batch(problems=20, seed=612, amax=5000)
    first = run_batch(lib, probs)
    lib.set_debug(3, 1)
    second = run_batch(lib, probs)
    for (x1, z1, c1), (x2, z2, c2), (a, b) in zip(first, second, probs):
        assert np.array_equal(x1, x2) and np.array_equal(z1, z2)
        check(x2, z2, c2, *oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple())[:4])


@pytest.mark.parametrize("leaf", [32, 64, 256])
def test_small_leaves_split_and_split_again(lib, oracle, leaf):
    # keys that vary on a few qubits only: children of a split still hold
    # many records and are split again at later positions
    from paper_2605_25974_gb300 import workloads as wl
    rng = np.random.default_rng(620 + leaf)
    probs = []
    for lo_q, na, nb in ((0, 900, 4), (250, 2500, 8), (490, 300, 1), (60, 1200, 3)):
        probs.append((sums(500, na, rng, wmax=6, lo_q=lo_q, hi_q=lo_q + 10),
                      sums(500, nb, rng, wmax=3, lo_q=lo_q, hi_q=lo_q + 10)))
    probs += wl.batch(problems=6, n=500, seed=621, amin=1, amax=3000)
    lib.set_debug(4, leaf)
    check_batch(lib, oracle, probs)


def test_one_key_problems_are_summed(lib, oracle):
    # A holds copies of one string s, B one string t: every product is s*t
    # (summed at the top); then copies of two strings, so that a split gives
    # children of one key each (summed below the split)
    from paper_2605_25974_gb300 import workloads as wl
    rng = np.random.default_rng(630)
    s = sums(500, 1, rng)
    t = sums(500, 1, rng)
    u = sums(500, 1, rng)
    a1 = wl.SumArrays(500, np.repeat(s.x, 5000, axis=1), np.repeat(s.z, 5000, axis=1),
                      wl.coeffs_normal(rng, 5000))
    two_x = np.concatenate([np.repeat(s.x, 3000, axis=1), np.repeat(u.x, 3000, axis=1)], axis=1)
    two_z = np.concatenate([np.repeat(s.z, 3000, axis=1), np.repeat(u.z, 3000, axis=1)], axis=1)
    perm = rng.permutation(6000)
    a2 = wl.SumArrays(500, two_x[:, perm].copy(), two_z[:, perm].copy(), wl.coeffs_normal(rng, 6000))
    small = wl.SumArrays(500, np.repeat(s.x, 40, axis=1), np.repeat(s.z, 40, axis=1), wl.coeffs_normal(rng, 40))
    tu = wl.SumArrays(500, np.concatenate([t.x, u.x], axis=1), np.concatenate([t.z, u.z], axis=1),
                      wl.coeffs_normal(rng, 2))
    probs = [(a1, t), (a2, t), (small, t), (a2, tu)]
    check_batch(lib, oracle, probs)
    lib.set_debug(4, 32)
    check_batch(lib, oracle, probs)


def test_keys_equal_in_their_first_window(lib, oracle):
    # strings built from three pieces: a head on qubits 0.., a middle on
    # qubits 200.. and a tail on qubits 400..499.  With few head and middle
    # patterns, many products agree on a leaf's 64-bit window (and on the
    # split codes) and differ only later, so the order comes from whole-key
    # comparisons.
    from paper_2605_25974_gb300 import workloads as wl
    rng = np.random.default_rng(640)
    probs = []
    for hq, mq, na, nb in ((1, 1, 700, 2), (3, 1, 700, 2), (2, 2, 1500, 1), (1, 1, 200, 8), (3, 2, 3000, 3)):
        head = sums(500, na, rng, wmax=hq, lo_q=0, hi_q=hq)
        mid = sums(500, na, rng, wmax=mq, lo_q=200, hi_q=200 + mq)
        tail = sums(500, na, rng, wmax=8, lo_q=400, hi_q=500)
        a = wl.SumArrays(500, head.x | mid.x | tail.x, head.z | mid.z | tail.z, head.c)
        bh = sums(500, nb, rng, wmax=hq, lo_q=0, hi_q=hq)
        bm = sums(500, nb, rng, wmax=mq, lo_q=200, hi_q=200 + mq)
        bt = sums(500, nb, rng, wmax=4, lo_q=400, hi_q=500)
        probs.append((a, wl.SumArrays(500, bh.x | bm.x | bt.x, bh.z | bm.z | bt.z, bh.c)))
    check_batch(lib, oracle, probs)
    lib.set_debug(4, 64)
    check_batch(lib, oracle, probs)


def test_empty_operands_and_tiny_problems(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    rng = np.random.default_rng(650)
    a = sums(300, 50, rng)
    b = sums(300, 3, rng)
    empty = wl.SumArrays(300, a.x[:, :0].copy(), a.z[:, :0].copy(), a.c[:0].copy())
    one_a = wl.SumArrays(300, a.x[:, :1].copy(), a.z[:, :1].copy(), a.c[:1].copy())
    one_b = wl.SumArrays(300, b.x[:, :1].copy(), b.z[:, :1].copy(), b.c[:1].copy())
    probs = [(a, b), (empty, b), (a, empty), (one_a, one_b), (empty, empty), (one_a, b)]
    for (pa, pb), (x, z, c) in zip(probs, run_batch(lib, probs)):
        ox, oz, oc, oabs, _ = oracle.multiply_canonical(300, pa.as_tuple(), pb.as_tuple())
        assert x.shape[1] == ox.shape[1]
        if ox.shape[1]:
            check(x, z, c, ox, oz, oc, oabs)


def test_large_right_operand_takes_the_general_pipeline(lib, oracle):
    # one right operand above the kernel's 64 terms: the whole batch takes the
    # general pipeline, with the same results
    rng = np.random.default_rng(660)
    probs = [(sums(200, 400, rng), sums(200, 70, rng)), (sums(200, 900, rng), sums(200, 5, rng))]
    check_batch(lib, oracle, probs)


def test_plan_graph_replay_on_the_persistent_kernel(lib, oracle):
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    probs = wl.batch(problems=40, seed=670, amax=4000)
    As = [lib.PauliSum.from_arrays(a) for a, _ in probs]
    Bs = [lib.PauliSum.from_arrays(b) for _, b in probs]
    expect = [oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple()) for a, b in probs]

    def verify(outs):
        for (ox, oz, oc, oabs, _), o in zip(expect, outs):
            x, z, c, _ = o.export()
            check(x, z, c, ox, oz, oc, oabs, TOL32)

    plan = lib.BatchPlan(As, Bs, "fp32_fp64merge")
    verify(plan.outputs())
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.launch(stream=s)
    for _ in range(3):
        g.replay()
        torch.cuda.current_stream().wait_stream(s)
        verify(plan.outputs())
    plan.close()
    for t in As + Bs:
        t.close()


@pytest.mark.parametrize("leaf_cap,split_fan", [(256, 1), (0, 4), (512, 3)])
def test_batch_tuning_sizes(lib, oracle, leaf_cap, split_fan):
    # the autotuner's sizes for the persistent kernel: other leaf capacities
    # and split fan-outs give the same sums
    from paper_2605_25974_gb300 import workloads as wl
    probs = wl.batch(problems=12, seed=680, amax=9000)
    lib.set_batch_tuning(leaf_cap, split_fan)
    try:
        check_batch(lib, oracle, probs)
    finally:
        lib.set_batch_tuning(0, 0)
    for bad in ((31, 2), (4096, 2), (0, 9), (-2, 0)):
        with pytest.raises(lib.PaulibError, match="INVALID_ARG"):
            lib.set_batch_tuning(*bad)


def test_batch_knob_argument_checks(lib):
    for knob, value in ((3, 2), (3, -1), (4, 31), (4, 4096), (4, -5)):
        with pytest.raises(lib.PaulibError, match="INVALID_ARG"):
            lib.set_debug(knob, value)
