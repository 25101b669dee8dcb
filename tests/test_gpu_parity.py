"""GPU path vs the CPU oracle, element by element, through the C ABI.

Bars (bit-exact where the result is an integer fact):
  * keys, their order and raw phases: bit-exact;
  * FP64 coefficients: |c_gpu - c_oracle| <= 1e-12 * sum |contribution|,
    per real and imaginary part (the tolerance the method is held to);
  * FP32-product modes: |c_gpu - c_oracle| <= TOL32 * sum |contribution|,
    TOL32 derived in fp32_tolerance() below.
"""
import numpy as np
import pytest

from conftest import keys_as_tuples

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def fp32_tolerance():
    # Inputs rounded to FP32 (2 roundings, rel. 2^-24 each), a complex product
    # with one FMA per part (<= 2 roundings of 2^-24 on terms bounded by
    # |c_a||c_b|), then an FP64 or compensated merge (negligible): per part
    # |error| <= ~6 * 2^-24 * |c_a||c_b| summed over contributions.  Use 8 ulps.
    return 8 * 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2605_25974_gb300 import paulib
    from paper_2605_25974_gb300.build import build
    build()
    torch.cuda.init()
    return paulib


def gpu_sum(lib, s):
    return lib.PauliSum.from_arrays(s)


def check_canonical(gx, gz, gc, ox, oz, oc, oabs, tol=TOL64):
    assert gx.shape == ox.shape, (gx.shape, ox.shape)
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz)
    err = np.maximum(np.abs(gc.real - oc.real), np.abs(gc.imag - oc.imag))
    bad = err > tol * oabs
    assert not bad.any(), "max rel err %.3g at %d terms" % (float(np.max(err / oabs)), int(bad.sum()))


def run_canonical(lib, a, b, precision="fp64"):
    with gpu_sum(lib, a) as ga, gpu_sum(lib, b) as gb:
        with lib.multiply(ga, gb, precision) as gc:
            assert gc.is_canonical
            x, z, c, k = gc.export()
    assert not k.any()
    return x, z, c


# ------------------------------------------------------------------ configurations

def test_tiny_n20_canonical(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    a, b = wl.tiny()
    x, z, c = run_canonical(lib, a, b)
    check_canonical(x, z, c, *oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple())[:4])


def test_tiny_n20_raw_bit_exact_keys_and_phases(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    a, b = wl.tiny()
    with gpu_sum(lib, a) as ga, gpu_sum(lib, b) as gb, lib.multiply(ga, gb, canonical=False) as gr:
        assert gr.n_terms == a.m * b.m and not gr.is_canonical
        x, z, c, k = gr.export()
    ox, oz, oc, ok = oracle.multiply_raw(a.n, a.as_tuple(), b.as_tuple())
    assert np.array_equal(x, ox) and np.array_equal(z, oz) and np.array_equal(k, ok)
    # c_a * c_b: the GPU contracts one multiply-add, the oracle does not
    bound = 4 * 2.0 ** -53 * np.abs(np.repeat(b.c, a.m)) * np.abs(np.tile(a.c, b.m))
    assert np.all(np.abs(c.real - oc.real) <= bound) and np.all(np.abs(c.imag - oc.imag) <= bound)


@pytest.mark.parametrize("n,m", [(100, 700), (200, 400), (64, 500), (20, 900)])
def test_jw_hh_scaled(lib, oracle, n, m):
    # Jordan-Wigner-shaped H*H (the duplicate-heavy workload), scaled so the
    # oracle finishes in seconds; several leaf ranges, splits and a heavy
    # identity key (m contributions).
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=n, m=m, seed=1000 + n)
    x, z, c = run_canonical(lib, h, h)
    ox, oz, oc, oabs, ocnt = oracle.multiply_canonical(n, h.as_tuple(), h.as_tuple())
    check_canonical(x, z, c, ox, oz, oc, oabs)
    assert ocnt.max() == m  # identity term


@pytest.mark.parametrize("n,m", [(100, 700), (200, 400), (20, 900), (30, 60)])
def test_same_operand_symmetric_path(lib, oracle, n, m):
    # multiply(H, H) with one handle: only pairs i <= j are generated, each
    # off-diagonal pair counted twice or cancelled by its commutation sign.
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=n, m=m, seed=2000 + n)
    ox, oz, oc, oabs, _ = oracle.multiply_canonical(n, h.as_tuple(), h.as_tuple())
    for prec, tol in (("fp64", TOL64), ("fp32_fp64merge", fp32_tolerance())):
        with gpu_sum(lib, h) as g, lib.multiply(g, g, prec) as gc:
            x, z, c, _ = gc.export()
        check_canonical(x, z, c, ox, oz, oc, oabs, tol=tol)


def test_same_operand_with_repeats_and_phases(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(31)
    n = 70
    ux, uz = wl.weighted_random(rng, n, 300, 1, 10)
    idx = rng.integers(0, 300, 2500)
    s = wl.SumArrays(n, ux[:, idx].copy(), uz[:, idx].copy(), wl.coeffs_normal(rng, 2500),
                     rng.integers(0, 4, 2500).astype(np.uint8))
    with gpu_sum(lib, s) as g, lib.multiply(g, g) as gc:
        x, z, c, _ = gc.export()
    check_canonical(x, z, c, *oracle.multiply_canonical(n, s.as_tuple(), s.as_tuple())[:4])


@pytest.mark.parametrize("n,ma,mb", [(500, 3000, 7), (500, 16, 8), (130, 1000, 33), (1024, 300, 5),
                                     (65, 2500, 3)])
def test_random_weighted_products(lib, oracle, n, ma, mb):
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(7 * n + ma)
    ax, az = wl.weighted_random(rng, n, ma, 1, min(n, 32))
    bx, bz = wl.weighted_random(rng, n, mb, 1, min(n, 32))
    a = wl.SumArrays(n, ax, az, wl.coeffs_loguniform(rng, ma))
    b = wl.SumArrays(n, bx, bz, wl.coeffs_loguniform(rng, mb))
    x, z, c = run_canonical(lib, a, b)
    check_canonical(x, z, c, *oracle.multiply_canonical(n, a.as_tuple(), b.as_tuple())[:4])


def test_single_string_products_bit_exact(lib, oracle):
    # A times single strings with coefficient exactly 1 (the streaming
    # workload's shape): every coefficient is +-c or +-ic of one input, exactly.
    from paper_2605_25974_gb300 import workloads as wl
    a, singles = wl.stream(m=20000, strings=3)
    for s in singles:
        x, z, c = run_canonical(lib, a, s)
        ox, oz, oc, oabs, ocnt = oracle.multiply_canonical(a.n, a.as_tuple(), s.as_tuple())
        assert np.array_equal(x, ox) and np.array_equal(z, oz)
        assert np.array_equal(c.view(np.uint64), oc.view(np.uint64))
        assert x.shape[1] == a.m


# ------------------------------------------------------------------ edge cases

def test_empty_operands(lib):
    from paper_2605_25974_gb300 import workloads as wl
    a, b = wl.tiny()
    e = wl.SumArrays(a.n, a.x[:, :0].copy(), a.z[:, :0].copy(), a.c[:0].copy())
    with gpu_sum(lib, e) as ge, gpu_sum(lib, b) as gb:
        for l, r in ((ge, gb), (gb, ge), (ge, ge)):
            with lib.multiply(l, r) as gc:
                assert gc.n_terms == 0 and gc.is_canonical
            with lib.multiply(l, r, canonical=False) as gr:
                assert gr.n_terms == 0
        with lib.compress(ge) as gc:
            assert gc.n_terms == 0


def test_one_by_one_and_n1(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    for n in (1, 2, 63, 64):
        a, b = wl.tiny(seed_a=3, seed_b=4, n=n, m=1)
        x, z, c = run_canonical(lib, a, b)
        check_canonical(x, z, c, *oracle.multiply_canonical(n, a.as_tuple(), b.as_tuple())[:4])
    # n = 1: all 16 letter pairs at once
    from conftest import parse_strings
    _, x1, z1 = parse_strings(list("IXYZ"))
    s = wl.SumArrays(1, x1, z1, np.array([1 + 2j, 3 - 1j, -2 + 0.5j, 0.25j]))
    x, z, c = run_canonical(lib, s, s)
    check_canonical(x, z, c, *oracle.multiply_canonical(1, s.as_tuple(), s.as_tuple())[:4])


def test_all_products_identical_heavy_key(lib, oracle):
    # Every product has the same string: the canonical form is one term whose
    # coefficient collects all contributions (a range with one repeated key
    # far beyond the shared-memory leaf size).
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(55)
    n = 100
    x1, z1 = wl.weighted_random(rng, n, 1, 1, n)
    ma = 20000
    a = wl.SumArrays(n, np.repeat(x1, ma, axis=1), np.repeat(z1, ma, axis=1), wl.coeffs_normal(rng, ma))
    b = wl.SumArrays(n, x1.copy(), z1.copy(), np.array([0.5 - 0.25j]))
    x, z, c = run_canonical(lib, a, b)
    assert x.shape[1] == 1 and not x.any() and not z.any()  # P*P = I
    check_canonical(x, z, c, *oracle.multiply_canonical(n, a.as_tuple(), b.as_tuple())[:4])


def test_half_heavy_half_distinct(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(56)
    n = 200
    hx, hz = wl.weighted_random(rng, n, 1, 1, 20)
    rx, rz = wl.weighted_random(rng, n, 6000, 1, 20)
    x = np.concatenate([np.repeat(hx, 6000, axis=1), rx], axis=1)
    z = np.concatenate([np.repeat(hz, 6000, axis=1), rz], axis=1)
    perm = rng.permutation(12000)
    a = wl.SumArrays(n, x[:, perm].copy(), z[:, perm].copy(), wl.coeffs_loguniform(rng, 12000))
    b = wl.SumArrays(n, *wl.weighted_random(rng, n, 3, 1, 20), wl.coeffs_loguniform(rng, 3))
    xx, zz, cc = run_canonical(lib, a, b)
    check_canonical(xx, zz, cc, *oracle.multiply_canonical(n, a.as_tuple(), b.as_tuple())[:4])


def test_compress_with_phases_and_duplicates(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(77)
    for n, m in ((30, 5000), (300, 9000)):
        ux, uz = wl.weighted_random(rng, n, 700, 1, 12)
        idx = rng.integers(0, 700, m)
        s = wl.SumArrays(n, ux[:, idx].copy(), uz[:, idx].copy(), wl.coeffs_normal(rng, m),
                         rng.integers(0, 4, m).astype(np.uint8))
        with gpu_sum(lib, s) as g, lib.compress(g) as gc:
            x, z, c, _ = gc.export()
        check_canonical(x, z, c, *oracle.compress(n, s.as_tuple())[:4])


def test_raw_then_compress_equals_canonical(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=40, m=300, seed=9)
    with gpu_sum(lib, h) as g:
        with lib.multiply(g, g, canonical=False) as raw, lib.compress(raw) as c1, lib.multiply(g, g) as c2:
            x1, z1, cc1, _ = c1.export()
            x2, z2, cc2, _ = c2.export()
    ox, oz, oc, oabs, _ = oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())
    check_canonical(x1, z1, cc1, ox, oz, oc, oabs)
    check_canonical(x2, z2, cc2, ox, oz, oc, oabs)


def test_errors(lib):
    from paper_2605_25974_gb300 import workloads as wl
    a, b = wl.tiny()
    bad = a.x.copy()
    bad[0, 0] |= np.uint64(1) << np.uint64(25)  # qubit 25 >= n = 20
    with pytest.raises(lib.PaulibError, match="TAIL_BITS"):
        lib.PauliSum.create(a.n, bad, a.z, a.c)
    c2, _ = wl.tiny(n=21)
    with gpu_sum(lib, a) as ga, gpu_sum(lib, c2) as gc:
        with pytest.raises(lib.PaulibError, match="QUBIT_MISMATCH"):
            lib.multiply(ga, gc)
        with pytest.raises(lib.PaulibError, match="INVALID_ARG"):
            lib.multiply(ga, ga, precision=7)


# ------------------------------------------------------------------ precision modes

@pytest.mark.parametrize("mode", ["fp32_fp64merge", "fp32_twosum"])
def test_mixed_precision_modes(lib, oracle, mode):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=100, m=500, seed=4)
    x, z, c = run_canonical(lib, h, h, mode)
    ox, oz, oc, oabs, _ = oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())
    check_canonical(x, z, c, ox, oz, oc, oabs, tol=fp32_tolerance())


# ------------------------------------------------------------------ batched

def test_batched_matches_per_problem_oracle(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    probs = wl.batch(problems=12, amax=3000)
    As = [gpu_sum(lib, a) for a, _ in probs]
    Bs = [gpu_sum(lib, b) for _, b in probs]
    outs = lib.multiply_batched(As, Bs, "fp64")
    for (a, b), o in zip(probs, outs):
        x, z, c, _ = o.export()
        check_canonical(x, z, c, *oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple())[:4])
    for s in As + Bs + outs:
        s.close()


def test_batch_plan_relaunch_and_graph_replay(lib, oracle):
    # A prepared plan relaunched (and replayed from a captured CUDA graph)
    # gives the same canonical outputs as the oracle, problem by problem.
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    probs = wl.batch(problems=9, amax=2000)
    probs.append((probs[0][0], wl.SumArrays(500, probs[0][1].x[:, :0].copy(), probs[0][1].z[:, :0].copy(),
                                            probs[0][1].c[:0].copy())))  # an empty problem
    As = [gpu_sum(lib, a) for a, _ in probs]
    Bs = [gpu_sum(lib, b) for _, b in probs]
    expect = [oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple()) for a, b in probs]

    def check(outs):
        for (ox, oz, oc, oabs, _), o in zip(expect, outs):
            x, z, c, _ = o.export()
            check_canonical(x, z, c, ox, oz, oc, oabs)

    plan = lib.BatchPlan(As, Bs, "fp64")
    check(plan.outputs())              # the run made while preparing
    plan.launch()
    check(plan.outputs())              # a plain relaunch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.launch(stream=s)
    for _ in range(2):
        g.replay()
        torch.cuda.current_stream().wait_stream(s)
        check(plan.outputs())
    plan.close()
    for t in As + Bs:
        t.close()


@pytest.mark.parametrize("mode", ["fp32_fp64merge", "fp32_twosum"])
def test_batched_mixed_precision(lib, oracle, mode):
    from paper_2605_25974_gb300 import workloads as wl
    probs = wl.batch(problems=6, amax=1500)
    As = [gpu_sum(lib, a) for a, _ in probs]
    Bs = [gpu_sum(lib, b) for _, b in probs]
    outs = lib.multiply_batched(As, Bs, mode)
    for (a, b), o in zip(probs, outs):
        x, z, c, _ = o.export()
        check_canonical(x, z, c, *oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple())[:4],
                        tol=fp32_tolerance())
    for s in As + Bs + outs:
        s.close()


def test_export_to_pinned_host_memory(lib, oracle):
    # page-locked host outputs are written by the export kernel directly;
    # pageable ones go through a device staging copy; both equal the device
    # export and the oracle
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=100, m=700, seed=11)
    with lib.PauliSum.from_arrays(h) as g, lib.multiply(g, g, "fp64") as o:
        W, U = o.words, o.n_terms
        dx = torch.empty((W, U), dtype=torch.int64, device="cuda")
        dz = torch.empty_like(dx)
        dc = torch.empty((U, 2), dtype=torch.float64, device="cuda")
        o.export(dx, dz, dc, None)
        px = torch.empty((W, U), dtype=torch.int64).pin_memory()
        pz = torch.empty((W, U), dtype=torch.int64).pin_memory()
        pc = torch.empty((U, 2), dtype=torch.float64).pin_memory()
        pk = torch.empty(U, dtype=torch.uint8).pin_memory()
        o.export(px, pz, pc, pk)
        nx, nz, nc, nk = o.export()
    torch.cuda.synchronize()
    assert np.array_equal(px.numpy().view(np.uint64), dx.cpu().numpy().view(np.uint64))
    assert np.array_equal(pz.numpy().view(np.uint64), nz)
    assert np.array_equal(pc.numpy().view(np.uint64), dc.cpu().numpy().view(np.uint64))
    assert np.array_equal(pc.numpy(), np.stack([nc.real, nc.imag], 1)) and not pk.numpy().any()
    ox, oz, oc, oabs, _ = oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())
    assert np.array_equal(nx, ox) and np.array_equal(nz, oz)


@pytest.mark.parametrize("m", [1000, 1001, 2])
def test_export_pinned_even_and_odd_counts(lib, m):
    # page-locked outputs written by the export kernel, even and odd term counts
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    rng = np.random.default_rng(m)
    x, z = wl.weighted_random(rng, 130, m, 1, 130)
    s = wl.SumArrays(130, x, z, wl.coeffs_loguniform(rng, m))
    with lib.PauliSum.from_arrays(s) as g:
        W = g.words
        px = torch.empty((W, m), dtype=torch.int64).pin_memory()
        pz = torch.empty((W, m), dtype=torch.int64).pin_memory()
        pc = torch.empty((m, 2), dtype=torch.float64).pin_memory()
        g.export(px, pz, pc, None)
        nx, nz, nc, _ = g.export()
    torch.cuda.synchronize()
    assert np.array_equal(px.numpy().view(np.uint64), nx) and np.array_equal(pz.numpy().view(np.uint64), nz)
    assert np.array_equal(nx, s.x) and np.array_equal(nz, s.z) and np.array_equal(nc, s.c)
    assert np.array_equal(pc.numpy()[:, 0], s.c.real) and np.array_equal(pc.numpy()[:, 1], s.c.imag)


@pytest.mark.parametrize("n,ma,mb,phases", [(100, 300, 37, False), (200, 129, 33, True), (500, 257, 31, False),
                                            (1024, 131, 45, True), (128, 127, 32, False), (65, 1, 1, True),
                                            (256, 130, 1, False)])
def test_raw_outer_product_every_word_width(lib, oracle, n, ma, mb, phases):
    # The tiled raw kernel (128 left terms per CTA x 32 right terms, keys
    # staged per warp) at 2, 4, 8 and 16 padded words per half, with ragged
    # last tiles in both directions (|A| not a multiple of 128, |B| not of
    # 32) and operand phases: keys and phases bit-exact, c_a*c_b within the
    # one-FMA bound, against the oracle's qubit-by-qubit products.
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(5 * n + ma)
    ax, az = wl.weighted_random(rng, n, ma, 1, min(n, 40))
    bx, bz = wl.weighted_random(rng, n, mb, 1, min(n, 40))
    ka = rng.integers(0, 4, ma).astype(np.uint8) if phases else None
    kb = rng.integers(0, 4, mb).astype(np.uint8) if phases else None
    a = wl.SumArrays(n, ax, az, wl.coeffs_normal(rng, ma), ka)
    b = wl.SumArrays(n, bx, bz, wl.coeffs_normal(rng, mb), kb)
    with gpu_sum(lib, a) as ga, gpu_sum(lib, b) as gb, lib.multiply(ga, gb, canonical=False) as gr:
        assert gr.n_terms == ma * mb and not gr.is_canonical
        x, z, c, k = gr.export()
    ox, oz, oc, ok = oracle.multiply_raw(n, a.as_tuple(), b.as_tuple())
    assert np.array_equal(x, ox) and np.array_equal(z, oz) and np.array_equal(k, ok)
    bound = 4 * 2.0 ** -53 * np.abs(np.repeat(b.c, ma)) * np.abs(np.tile(a.c, mb))
    assert np.all(np.abs(c.real - oc.real) <= bound) and np.all(np.abs(c.imag - oc.imag) <= bound)
