"""Full-size parity: the benchmark's workloads at their full sizes, run the way
bench.py times them (two handles holding H, FP64, canonical output; batched
products as a prepared plan replayed from a CUDA graph), and checked

  * on sampled outputs the oracle computes one by one from the definition
    (coefficient of a given string in A*B: PauLIB Sec. IV-C with the
    single-qubit table of Sec. III-A),
  * by properties that hold at any size: keys strictly increasing (Sec.
    III-H), every sampled pair product present, the identity coefficient of
    H*H equal to sum_j c_j^2,
  * and, where the oracle finishes in seconds at full size (the streaming
    workload's single-string products, sampled batched problems), element by
    element.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
SIGN = -(1 << 63)  # flips the top bit: unsigned word order as signed int64 order


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2605_25974_gb300 import paulib
    from paper_2605_25974_gb300.build import build
    build()
    torch.cuda.init()
    return paulib


def export_device(gc, W):
    """Exports a device sum into device tensors: keys (2W, U) as order-
    preserving int64, coefficients (U,) complex128."""
    import torch
    U = gc.n_terms
    x = torch.empty((W, U), dtype=torch.int64, device="cuda")
    z = torch.empty_like(x)
    c = torch.empty((U, 2), dtype=torch.float64, device="cuda")
    gc.export(x, z, c, None)
    torch.cuda.synchronize()
    return torch.cat([x, z]) ^ SIGN, torch.view_as_complex(c)


def lex_less(a, b):
    """Column-wise lexicographic a < b for (words, k) int64 tensors."""
    import torch
    neq = a != b
    first = neq.to(torch.int32).argmax(0, keepdim=True)  # first differing word
    return neq.any(0) & (a.gather(0, first) < b.gather(0, first))[0]


def assert_strictly_increasing(keys, chunk=1 << 25):
    U = keys.shape[1]
    for s in range(0, max(U - 1, 0), chunk):
        e = min(U - 1, s + chunk)
        assert bool(lex_less(keys[:, s:e], keys[:, s + 1:e + 1]).all()), "keys not strictly increasing near %d" % s


def find_rows(keys, q):
    """Index of each query column of q in the sorted keys (or -1)."""
    import torch
    U = keys.shape[1]
    S = q.shape[1]
    lo = torch.zeros(S, dtype=torch.int64, device=keys.device)
    hi = torch.full((S,), U, dtype=torch.int64, device=keys.device)
    for _ in range(int(np.ceil(np.log2(max(U, 2)))) + 2):
        mid = torch.minimum((lo + hi) // 2, torch.full_like(lo, U - 1))
        go = lo < hi
        less = lex_less(keys[:, mid], q) & go
        lo = torch.where(less, mid + 1, lo)
        hi = torch.where(go & ~less, mid, hi)
    pos = torch.minimum(lo, torch.full_like(lo, U - 1))
    hit = (keys[:, pos] == q).all(0) & (lo < U)
    return torch.where(hit, pos, torch.full_like(pos, -1))


def to_words(t):
    return (t ^ SIGN).cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("n,m,seed", [(100, 20000, 301), (200, 30000, 401)])
def test_jw_hh_full_size(lib, oracle, n, m, seed):
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=n, m=m, seed=seed)
    W = h.x.shape[0]
    with lib.PauliSum.from_arrays(h) as ga, lib.PauliSum.from_arrays(h) as gb, lib.multiply(ga, gb, "fp64") as gc:
        assert gc.is_canonical and 0 < gc.n_terms <= m * m
        keys, c = export_device(gc, W)
    U = keys.shape[1]
    assert_strictly_increasing(keys)

    # the identity (all-zero key, the smallest) collects c_j^2 from every j
    assert bool((keys[:, 0] == SIGN).all())
    ident = np.sum(h.c * h.c)
    scale = np.sum(np.abs(h.c) ** 2)
    got = complex(c[0].item())
    assert abs(got.real - ident.real) <= TOL64 * scale and abs(got.imag - ident.imag) <= TOL64 * scale

    # sampled outputs: each coefficient from the definition
    rng = np.random.default_rng(seed)
    idx = np.unique(rng.integers(0, U, size=160))
    qk = to_words(keys[:, torch.from_numpy(idx).cuda()])
    oc, oabs, ocnt = oracle.query_product_coeffs(n, h.as_tuple(), h.as_tuple(), qk[:W], qk[W:])
    assert (ocnt > 0).all(), "an output string is not a product of the operands"
    gcs = c[torch.from_numpy(idx).cuda()].cpu().numpy()
    err = np.maximum(np.abs(gcs.real - oc.real), np.abs(gcs.imag - oc.imag))
    assert (err <= TOL64 * oabs).all(), float(np.max(err / oabs))

    # sampled pair products: every one's string is in the output
    pi = rng.integers(0, m, size=300)
    pj = rng.integers(0, m, size=300)
    q = np.zeros((2 * W, len(pi)), np.uint64)
    for t, (i, j) in enumerate(zip(pi, pj)):
        xo, zo, _ = oracle.string_product(n, h.x[:, i], h.z[:, i], h.x[:, j], h.z[:, j])
        q[:W, t], q[W:, t] = xo, zo
    qt = torch.from_numpy(q.view(np.int64)).cuda() ^ SIGN
    assert bool((find_rows(keys, qt) >= 0).all()), "a pair product is missing from the output"


def test_stream_full_size_single_strings(lib, oracle):
    # the streaming workload: the 1,000,000-term n=500 sum times single
    # strings with coefficient 1; every output coefficient is exactly +-c or
    # +-ic of one input, so the comparison is bit for bit
    from paper_2605_25974_gb300 import workloads as wl
    a, singles = wl.stream(strings=2)
    with lib.PauliSum.from_arrays(a) as ga:
        for s in singles:
            with lib.PauliSum.from_arrays(s) as gs, lib.multiply(ga, gs, "fp64") as gc:
                x, z, c, _ = gc.export()
            ox, oz, oc, _, ocnt = oracle.multiply_canonical(a.n, a.as_tuple(), s.as_tuple())
            assert x.shape[1] == a.m and (ocnt == 1).all()
            assert np.array_equal(x, ox) and np.array_equal(z, oz)
            assert np.array_equal(c.view(np.uint64), oc.view(np.uint64))


def test_batched_full_size_graph_replay(lib, oracle):
    # the batching workload at full size (4,096 problems), as a prepared plan
    # replayed from a CUDA graph with FP32 products and FP64 merge; sampled
    # problems compared element by element with the oracle, every problem
    # checked for key order
    import torch
    from paper_2605_25974_gb300 import workloads as wl
    probs = wl.batch(problems=4096)
    As = [lib.PauliSum.from_arrays(a) for a, _ in probs]
    Bs = [lib.PauliSum.from_arrays(b) for _, b in probs]
    plan = lib.BatchPlan(As, Bs, "fp32_fp64merge")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.launch(stream=s)
    g.replay()
    torch.cuda.current_stream().wait_stream(s)
    outs = plan.outputs()
    tol = 8 * 2.0 ** -24
    rng = np.random.default_rng(4096)
    for q in sorted(set(rng.integers(0, len(probs), size=24).tolist()) | {int(np.argmax([a.m for a, _ in probs]))}):
        a, b = probs[q]
        x, z, c, _ = outs[q].export()
        ox, oz, oc, oabs, _ = oracle.multiply_canonical(a.n, a.as_tuple(), b.as_tuple())
        assert np.array_equal(x, ox) and np.array_equal(z, oz), "problem %d" % q
        err = np.maximum(np.abs(c.real - oc.real), np.abs(c.imag - oc.imag))
        assert (err <= tol * oabs).all(), "problem %d: %.3g" % (q, float(np.max(err / oabs)))
    assert all(o.n_terms <= a.m * b.m for o, (a, b) in zip(outs, probs))
    # every problem's output, not only the sampled ones: keys strictly
    # increasing (a canonical sum holds each string once, in key order), and
    # for the problems of at most 4,096 products the keys equal the distinct
    # products a_i XOR b_j sorted (numpy's row order is the key order: x
    # words, then z words, word 0 most significant)
    for q, o in enumerate(outs):
        x, z, c, _ = o.export()
        K = np.concatenate([x, z], axis=0).T
        if len(K) > 1:
            D = K[1:] != K[:-1]
            first = np.argmax(D, axis=1)
            rows = np.arange(len(K) - 1)
            assert D.any(axis=1).all() and (K[1:][rows, first] > K[:-1][rows, first]).all(), "problem %d" % q
        a, b = probs[q]
        if a.m * b.m <= 4096:
            ka = np.concatenate([a.x, a.z], axis=0).T
            kb = np.concatenate([b.x, b.z], axis=0).T
            prod = np.unique((ka[:, None, :] ^ kb[None, :, :]).reshape(-1, ka.shape[1]), axis=0)
            assert np.array_equal(K, prod), "problem %d" % q
    plan.close()
    for t in As + Bs:
        t.close()
