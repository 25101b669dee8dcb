"""Clifford gate application and the Pauli rotation step (Sec. III-B) on the
GPU against the CPU oracle, through the C ABI.  Keys, their order and term
counts bit-exact; coefficients of Clifford images exact (a sign change);
rotation coefficients within 1e-12 * sum |contribution| (FP64 merge)."""
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


def random_terms(rng, n, m, with_phase=False):
    from paper_2605_25974_gb300 import workloads as wl
    x, z = wl.weighted_random(rng, n, m, 1, n)
    c = wl.coeffs_loguniform(rng, m)
    k = rng.integers(0, 4, m).astype(np.uint8) if with_phase else None
    return wl.SumArrays(n, x, z, c, k)


def random_gates(rng, n, count):
    gates = []
    for _ in range(count):
        g = ["h", "s", "cnot", "cz"][rng.integers(0, 4)]
        q1 = int(rng.integers(0, n))
        q2 = int(rng.integers(0, n - 1))
        q2 = q2 + 1 if q2 >= q1 else q2
        gates.append((g, q1, q2))
    return gates


@pytest.mark.parametrize("n,m,ng", [(5, 40, 1), (70, 3000, 25), (130, 5000, 60), (500, 2000, 200), (64, 700, 9)])
def test_clifford_list_vs_oracle(lib, oracle, n, m, ng):
    rng = np.random.default_rng(11 * n + ng)
    s = random_terms(rng, n, m, with_phase=True)
    gates = random_gates(rng, n, ng)
    with lib.PauliSum.from_arrays(s) as g:
        lib.apply_clifford(g, gates)
        assert not g.is_canonical or ng == 0
        x, z, c, k = g.export()
    # oracle: gate by gate, phases folded in at the first gate
    ox, oz, oc = s.x, s.z, s.c
    ok = s.k
    for gate, q1, q2 in gates:
        ox, oz, oc = oracle.apply_clifford(n, (ox, oz, oc, ok), gate, q1, q2)
        ok = None
    assert np.array_equal(x, ox) and np.array_equal(z, oz)
    # the GPU keeps the term's phase byte and moves only the sign into c
    ik = np.array([1, 1j, -1, -1j])[k]
    assert np.array_equal((c * ik).view(np.uint64), oc.view(np.uint64)) or np.allclose(c * ik, oc, atol=0, rtol=0)


ONE_WORD_LISTS = [
    (500, [("h", 3, 0)]), (500, [("s", 200, 0)]), (500, [("cnot", 130, 191)]), (500, [("cz", 64, 127)]),
    (500, [("h", 256, 0), ("s", 256, 0), ("cnot", 256, 300), ("cz", 319, 257), ("h", 300, 0), ("s", 319, 0)]),
    (130, [("s", 129, 0), ("h", 128, 0), ("cnot", 128, 129), ("cz", 129, 128)]),  # the last, partial word
    (64, [("h", 0, 0), ("cz", 0, 63), ("s", 63, 0), ("cnot", 63, 0)]),
]


@pytest.mark.parametrize("n,gates", ONE_WORD_LISTS)
def test_clifford_one_word_lists(lib, oracle, n, gates):
    # every qubit of the list in one 64-bit word: the kernel that reads and
    # writes only that word, the phase byte and the flipped coefficients.  The
    # product with a second sum afterwards checks the updated phase bases.
    rng = np.random.default_rng(n + len(gates))
    s = random_terms(rng, n, 3000, with_phase=True)
    b = random_terms(rng, n, 40)
    with lib.PauliSum.from_arrays(s) as g, lib.PauliSum.from_arrays(b) as gb:
        lib.apply_clifford(g, gates)
        x, z, c, k = g.export()
        with lib.multiply(g, gb, "fp64") as gp:
            px, pz, pc, _ = gp.export()
    ox, oz, oc = s.x, s.z, s.c
    ok = s.k
    for gate, q1, q2 in gates:
        ox, oz, oc = oracle.apply_clifford(n, (ox, oz, oc, ok), gate, q1, q2)
        ok = None
    assert np.array_equal(x, ox) and np.array_equal(z, oz)
    ik = np.array([1, 1j, -1, -1j])[k]
    assert np.array_equal(c * ik, oc)
    qx, qz, qc, qabs, _ = oracle.multiply_canonical(n, (ox, oz, oc), b.as_tuple())
    assert np.array_equal(px, qx) and np.array_equal(pz, qz)
    err = np.maximum(np.abs(pc.real - qc.real), np.abs(pc.imag - qc.imag))
    assert (err <= TOL64 * qabs).all()


def test_clifford_then_compress_is_canonical(lib, oracle):
    rng = np.random.default_rng(5)
    n = 100
    s = random_terms(rng, n, 4000)
    gates = random_gates(rng, n, 30)
    with lib.PauliSum.from_arrays(s) as g:
        lib.apply_clifford(g, gates)
        with lib.compress(g) as gc:
            x, z, c, _ = gc.export()
    ox, oz, oc = s.x, s.z, s.c
    for gate, q1, q2 in gates:
        ox, oz, oc = oracle.apply_clifford(n, (ox, oz, oc), gate, q1, q2)
    cx, cz, cc, cabs, _ = oracle.compress(n, (ox, oz, oc))
    assert np.array_equal(x, cx) and np.array_equal(z, cz)
    assert (np.abs(c - cc) <= TOL64 * cabs).all()


def test_clifford_errors(lib):
    from paper_2605_25974_gb300 import workloads as wl
    a, _ = wl.tiny()
    with lib.PauliSum.from_arrays(a) as g:
        for bad in ([("h", 20, 0)], [("cnot", 3, 3)], [(7, 1, 2)], [("cz", -1, 2)]):
            with pytest.raises(lib.PaulibError) as e:
                lib.apply_clifford(g, bad)
            assert "INVALID_ARG" in str(e.value)
        x0, z0, c0, _ = g.export()
        assert np.array_equal(x0, a.x)  # nothing changed


@pytest.mark.parametrize("n,m,theta,thr", [(6, 50, 0.37, 0.0), (100, 3000, 1.1, 0.0), (200, 5000, 0.2, 1e-4),
                                           (500, 2000, np.pi / 2, 0.0), (70, 4000, np.pi, 0.0), (64, 3000, -0.8, 1e-3)])
def test_rotation_vs_oracle(lib, oracle, n, m, theta, thr):
    rng = np.random.default_rng(13 * n + m)
    s = random_terms(rng, n, m, with_phase=True)
    # duplicates: the generator times some terms are other terms
    p = random_terms(rng, n, 1)
    px, pz = p.x[:, 0], p.z[:, 0]
    with lib.PauliSum.from_arrays(s) as g, lib.rotate(g, px, pz, theta, thr) as r:
        assert r.is_canonical
        x, z, c, _ = r.export()
    ox, oz, oc, oabs, _ = oracle.rotate(n, s.as_tuple(), px, pz, theta, thr)
    assert np.array_equal(x, ox) and np.array_equal(z, oz)
    err = np.maximum(np.abs(c.real - oc.real), np.abs(c.imag - oc.imag))
    assert (err <= TOL64 * np.maximum(oabs, 1e-300)).all(), float(np.max(err / np.maximum(oabs, 1e-300)))


@pytest.mark.parametrize("n,m,theta,thr,prec", [(5, 600, 0.4, 0.0, "fp64"), (70, 5000, 1.1, 0.0, "fp64"),
                                                 (130, 20000, -0.7, 1e-3, "fp64"), (500, 3000, 0.25, 0.0, "fp64"),
                                                 (1024, 900, 2.0, 0.0, "fp64"), (200, 8000, 0.9, 0.0, "fp32_fp64merge")])
def test_rotation_of_canonical_sum_merges(lib, oracle, n, m, theta, thr, prec):
    # a canonical input takes the merge path: the Q part stays sorted, only
    # the partners P Q are canonicalised, then the two lists are merged.  Half
    # of the terms are P times other terms, so many partners land on existing
    # keys; the oracle rotates the raw input directly.
    from paper_2605_25974_gb300 import workloads as wl
    rng = np.random.default_rng(7 * n + m)
    base = random_terms(rng, n, m // 2)
    p = random_terms(rng, n, 1)
    px, pz = p.x[:, 0], p.z[:, 0]
    shifted = wl.SumArrays(n, base.x ^ px[:, None], base.z ^ pz[:, None], wl.coeffs_loguniform(rng, m // 2))
    both = wl.SumArrays(n, np.concatenate([base.x, shifted.x], 1), np.concatenate([base.z, shifted.z], 1),
                        np.concatenate([base.c, shifted.c]))
    with lib.PauliSum.from_arrays(both) as g, lib.compress(g) as cg:
        assert cg.is_canonical
        with lib.rotate(cg, px, pz, theta, thr, prec) as r:
            assert r.is_canonical
            x, z, c, _ = r.export()
    ox, oz, oc, oabs, _ = oracle.rotate(n, both.as_tuple(), px, pz, theta, thr)
    assert np.array_equal(x, ox) and np.array_equal(z, oz)
    tol = TOL64 if prec == "fp64" else 8 * 2.0 ** -24 * 2
    err = np.maximum(np.abs(c.real - oc.real), np.abs(c.imag - oc.imag))
    assert (err <= tol * np.maximum(oabs, 1e-300)).all(), float(np.max(err / np.maximum(oabs, 1e-300)))


def test_rotation_of_canonical_sum_tiny_cases(lib, oracle):
    # one term, every term anti-commuting, and partners landing on other terms
    from conftest import parse_strings
    from paper_2605_25974_gb300 import workloads as wl
    cases = [(["XZ"], "ZI", 0.3), (["XI", "YI", "XZ"], "ZI", 0.8), (["IZ", "XZ", "YZ"], "ZZ", 1.3)]
    for strs, gen, theta in cases:
        n, x, z = parse_strings(strs)
        c = np.arange(1, len(strs) + 1).astype(np.complex128) * (1 + 0.5j)
        _, gx, gz = parse_strings([gen])
        s = wl.SumArrays(n, x, z, c)
        with lib.PauliSum.from_arrays(s) as g, lib.compress(g) as cg, lib.rotate(cg, gx[:, 0], gz[:, 0], theta) as r:
            rx, rz, rc, _ = r.export()
        ox, oz, oc, oabs, _ = oracle.rotate(n, s.as_tuple(), gx[:, 0], gz[:, 0], theta)
        assert np.array_equal(rx, ox) and np.array_equal(rz, oz)
        assert np.allclose(rc, oc, atol=1e-14, rtol=0)


def test_rotation_of_jw_hamiltonian_step(lib, oracle):
    # a propagation step on a Jordan-Wigner-shaped sum: many duplicates merge
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=60, m=3000, seed=77)
    px, pz = h.x[:, 5], h.z[:, 5]  # a generator drawn from the sum itself
    with lib.PauliSum.from_arrays(h) as g, lib.rotate(g, px, pz, 0.3, 0.0, "fp32_fp64merge") as r:
        x, z, c, _ = r.export()
    ox, oz, oc, oabs, _ = oracle.rotate(60, h.as_tuple(), px, pz, 0.3, 0.0)
    assert np.array_equal(x, ox) and np.array_equal(z, oz)
    assert (np.abs(c - oc) <= 8 * 2.0 ** -24 * 2 * oabs).all()


def test_rotation_empty_and_tail_bits(lib):
    from paper_2605_25974_gb300 import workloads as wl
    a, _ = wl.tiny()
    with lib.PauliSum.from_arrays(a) as g:
        bad = np.zeros(1, np.uint64)
        bad[0] = 1 << 40  # qubit 40 >= n = 20
        with pytest.raises(lib.PaulibError) as e:
            lib.rotate(g, bad, np.zeros(1, np.uint64), 0.5)
        assert "TAIL_BITS" in str(e.value)
        # identity generator: every term commutes, the result is the canonical input
        with lib.rotate(g, np.zeros(1, np.uint64), np.zeros(1, np.uint64), 0.7) as r, lib.compress(g) as cg:
            assert np.array_equal(r.export()[0], cg.export()[0])


@pytest.mark.parametrize("n,m", [(20, 1), (64, 1000), (200, 30000), (500, 100000)])
def test_pairwise_products_bit_exact(lib, oracle, n, m):
    rng = np.random.default_rng(n + m)
    a = random_terms(rng, n, m, with_phase=True)
    b = random_terms(rng, n, m, with_phase=True)
    with lib.PauliSum.from_arrays(a) as ga, lib.PauliSum.from_arrays(b) as gb, lib.multiply_pairwise(ga, gb) as o:
        assert o.n_terms == m and not o.is_canonical
        x, z, c, k = o.export()
    ox, oz, oc, ok = oracle.multiply_pairwise(n, a.as_tuple(), b.as_tuple())
    assert np.array_equal(x, ox) and np.array_equal(z, oz) and np.array_equal(k, ok)
    # c_a * c_b: the GPU contracts one multiply-add, the oracle does not
    bound = 4 * 2.0 ** -53 * np.abs(a.c) * np.abs(b.c)
    assert np.all(np.abs(c.real - oc.real) <= bound) and np.all(np.abs(c.imag - oc.imag) <= bound)


def test_pairwise_errors(lib):
    from paper_2605_25974_gb300 import workloads as wl
    a, b = wl.tiny()
    with lib.PauliSum.from_arrays(a) as ga, lib.PauliSum.from_arrays(b.subset(slice(0, 10))) as gb:
        with pytest.raises(lib.PaulibError) as e:
            lib.multiply_pairwise(ga, gb)
        assert "INVALID_ARG" in str(e.value)
