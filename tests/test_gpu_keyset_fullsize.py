"""Full-size key-set parity: every term of the GPU's canonical H*H compared
with the CPU oracle, one key range at a time.

The Jordan-Wigner-shaped H*H at n=100 with 20,000 terms (4e8 products, about
2e8 merged terms) is computed once on the GPU.  Range bounds are sorted keys
of a seeded sample of product pairs (numpy XOR of the words; neither side of
the comparison supplies them).  For each range the oracle's key-range,
multi-threaded canonical product gives the expected terms; the GPU sum is
exported slice by slice (the slice of range r starts where range r-1 ended),
so a missing or extra string anywhere shifts every later slice and fails.

Bars: keys and their order bit-exact, coefficients within 1e-12 *
sum |contribution| per part.  The n=200, 30,000-term product (9e8 products)
runs too when PAULIB_FULLSIZE_N200=1 (about seven minutes on 16 host cores).
"""
import os

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
    return paulib


def sample_bounds(a, b, nsamp, nranges, seed):
    rng = np.random.default_rng(seed)
    ia = rng.integers(0, a.m, nsamp)
    jb = rng.integers(0, b.m, nsamp)
    k = np.concatenate([a.x[:, ia] ^ b.x[:, jb], a.z[:, ia] ^ b.z[:, jb]], axis=0).T
    k = np.unique(k, axis=0)
    step = max(1, len(k) // nranges)
    return [k[q] for q in range(step, len(k), step)]


def check_every_term(lib, oracle, h, nranges, precision="fp64"):
    threads = max(1, os.cpu_count() or 1)
    bounds = sample_bounds(h, h, 200000, nranges, h.n)
    edges = [None] + bounds + [None]
    with lib.PauliSum.from_arrays(h) as ga, lib.PauliSum.from_arrays(h) as gb, \
            lib.multiply(ga, gb, precision) as gc:
        U = gc.n_terms
        start = 0
        worst = 0.0
        for lo, hi in zip(edges[:-1], edges[1:]):
            ox, oz, oc, oabs, ocnt = oracle.multiply_canonical_range(h.n, h.as_tuple(), h.as_tuple(), lo, hi,
                                                                     threads)
            u = ox.shape[1]
            assert start + u <= U, "the GPU sum has fewer terms than the oracle"
            gx, gz, gcf, _ = gc.export_range(start, u)
            assert np.array_equal(gx, ox) and np.array_equal(gz, oz), "keys differ in range at %d" % start
            err = np.maximum(np.abs(gcf.real - oc.real), np.abs(gcf.imag - oc.imag))
            assert np.all(err <= TOL64 * oabs), "coefficient beyond tolerance in range at %d" % start
            worst = max(worst, float(np.max(err / oabs)) if u else 0.0)
            start += u
        assert start == U, "the GPU sum has %d terms, the oracle %d" % (U, start)
    return U, worst


def test_jw_hh_n100_m20000_every_term(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=100, m=20000, seed=301)
    U, worst = check_every_term(lib, oracle, h, 24)
    assert U > 1.9e8
    print("n=100 H*H: %d terms, all keys equal, max rel coefficient error %.3g" % (U, worst))


@pytest.mark.skipif(os.environ.get("PAULIB_FULLSIZE_N200") != "1", reason="set PAULIB_FULLSIZE_N200=1")
def test_jw_hh_n200_m30000_every_term(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=200, m=30000, seed=401)
    U, worst = check_every_term(lib, oracle, h, 48)
    assert U > 4.4e8
    print("n=200 H*H: %d terms, all keys equal, max rel coefficient error %.3g" % (U, worst))
