"""Seeded generators: shapes, distributions and structure of the synthetic
workloads (no GPU)."""
import numpy as np

from paper_2605_25974_gb300 import workloads as wl


def popcount_rows(words):
    return np.array([sum(bin(int(w)).count("1") for w in col) for col in words.T])


def test_pack_unpack_roundtrip():
    rng = np.random.default_rng(0)
    for n in (1, 20, 64, 65, 200, 500):
        bits = rng.random((37, n)) < 0.3
        assert np.array_equal(wl.unpack_bits(wl.pack_bits(bits, n), n), bits)


def test_tiny_shape_and_determinism():
    a, b = wl.tiny()
    assert a.n == 20 and a.m == 64 and b.m == 64 and a.x.shape == (1, 64)
    a2, _ = wl.tiny()
    assert np.array_equal(a.x, a2.x) and np.array_equal(a.c, a2.c)
    assert not np.array_equal(a.x, b.x)
    assert not (a.x >> np.uint64(20)).any() and not (a.z >> np.uint64(20)).any()


def test_weighted_random_weights_and_distinctness():
    rng = wl.rng_for(3)
    x, z = wl.weighted_random(rng, 500, 2000, 1, 32)
    w = popcount_rows(x | z)
    assert w.min() >= 1 and w.max() <= 32
    assert len(wl._dedupe(x, z)) == 2000
    assert not (x[-1] >> np.uint64(500 - 448)).any()  # qubits >= 500 are zero


def test_jw_structure():
    h = wl.jw(n=100, m=3000, seed=11)
    assert h.m == 3000 and len(wl._dedupe(h.x, h.z)) == 3000
    xw = popcount_rows(h.x)
    assert set(np.unique(xw)) <= {0, 2, 4}            # Z-only, one-body, two-body
    assert (xw == 0).sum() == 100 + 300                # single Z on every qubit + 10% ZZ
    assert (xw == 2).sum() == 600                      # 20% one-body terms
    mags = np.abs(h.c)
    assert mags.min() >= 1e-6 * (1 - 1e-12) and mags.max() <= 1 + 1e-12


def test_stream_singles_have_unit_coefficient():
    a, singles = wl.stream(m=3000, strings=4)
    assert a.n == 500 and a.m == 3000 and len(singles) == 4
    for s in singles:
        assert s.m == 1 and s.c[0] == 1 + 0j
    w = popcount_rows(a.x | a.z)
    assert w.min() >= 1 and w.max() <= 500


def test_batch_sizes():
    probs = wl.batch(problems=20)
    for a, b in probs:
        assert 16 <= a.m <= 16384 and 1 <= b.m <= 8 and a.n == 500
        assert popcount_rows(a.x | a.z).max() <= 32
    again = wl.batch(problems=20)
    assert np.array_equal(again[2][0].x, probs[2][0].x) and np.array_equal(again[7][1].c, probs[7][1].c)


def test_grouping_workload():
    # random 500-qubit sums: every qubit uniform over {I, X, Y, Z}, distinct
    # strings, seeded by size
    for m in (200, 2000):
        h = wl.grouping(m)
        assert h.n == 500 and h.m == m and h.x.shape == (8, m)
        assert len(wl._dedupe(h.x, h.z)) == m
        assert np.array_equal(h.x, wl.grouping(m).x)
        assert not (h.x[-1] >> np.uint64(500 - 448)).any() and not (h.z[-1] >> np.uint64(500 - 448)).any()
        # letters: each of I, X, Y, Z on about a quarter of the qubits
        xb, zb = wl.unpack_bits(h.x, 500), wl.unpack_bits(h.z, 500)
        frac = [np.mean(~xb & ~zb), np.mean(xb & ~zb), np.mean(xb & zb), np.mean(~xb & zb)]
        assert all(abs(f - 0.25) < 0.02 for f in frac)
    assert not np.array_equal(wl.grouping(200).x[:, :10], wl.grouping(300).x[:, :10])
