"""Pins the CPU oracle to facts that do not come from the oracle itself:
the paper's Pauli matrices and stated products (Sec. III-A), Kronecker
products computed by numpy, the symplectic inner product (Sec. III-F),
closed forms and invariants of the Pauli algebra, and library sorting/summing.
"""
import itertools
import math

import numpy as np
import pytest

from conftest import LETTERS, keys_as_tuples, parse_strings, format_strings, read_golden


# The four Pauli matrices as printed in Sec. III-A.
MATS = {
    "I": np.array([[1, 0], [0, 1]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
}
IK = [1, 1j, -1, -1j]


def string_matrix(s):
    m = np.array([[1]], dtype=complex)
    for ch in s:
        m = np.kron(m, MATS[ch])
    return m


def all_strings(n):
    return ["".join(p) for p in itertools.product(LETTERS, repeat=n)]


def oracle_product_of_strings(oracle, sa, sb):
    n, xa, za = parse_strings([sa])
    _, xb, zb = parse_strings([sb])
    xo, zo, k = oracle.string_product(n, xa[:, 0], za[:, 0], xb[:, 0], zb[:, 0])
    return format_strings(n, xo.reshape(-1, 1), zo.reshape(-1, 1))[0], k


# ------------------------------------------------------------------ matrices

def test_paper_matrices_y_is_ixz():
    # Sec. III-A: Y = iXZ, P^2 = I, P Hermitian.
    assert np.allclose(MATS["Y"], 1j * MATS["X"] @ MATS["Z"])
    for m in MATS.values():
        assert np.allclose(m @ m, np.eye(2))
        assert np.allclose(m, m.conj().T)


def test_letter_table_matches_matrix_products(oracle):
    for a, b in itertools.product(range(4), repeat=2):
        c, k = oracle.letter_product(a, b)
        lhs = MATS[LETTERS[a]] @ MATS[LETTERS[b]]
        assert np.allclose(lhs, IK[k] * MATS[LETTERS[c]]), (LETTERS[a], LETTERS[b])


def test_paper_stated_products(oracle):
    rows = read_golden("paper_products.txt")
    assert len(rows) >= 13
    for sa, sb, sp, k in rows:
        prod, kk = oracle_product_of_strings(oracle, sa, sb)
        assert prod == sp and kk == int(k), (sa, sb, prod, kk)
        # and the golden row itself agrees with the matrices
        assert np.allclose(string_matrix(sa) @ string_matrix(sb), IK[int(k)] * string_matrix(sp))


def test_exhaustive_two_qubit_products_vs_kron(oracle):
    strs = all_strings(2)
    for sa, sb in itertools.product(strs, repeat=2):
        prod, k = oracle_product_of_strings(oracle, sa, sb)
        assert np.allclose(string_matrix(sa) @ string_matrix(sb), IK[k] * string_matrix(prod)), (sa, sb)


@pytest.mark.parametrize("n", [3, 4])
def test_random_products_vs_kron(oracle, n):
    rng = np.random.default_rng(7 + n)
    for _ in range(300):
        sa = "".join(rng.choice(list(LETTERS), n))
        sb = "".join(rng.choice(list(LETTERS), n))
        prod, k = oracle_product_of_strings(oracle, sa, sb)
        assert np.allclose(string_matrix(sa) @ string_matrix(sb), IK[k] * string_matrix(prod))


def test_multiword_product_matches_per_qubit_kron(oracle):
    # Strings longer than one 64-bit word: the product factorises over qubits,
    # so each qubit must follow the single-qubit matrix product.
    rng = np.random.default_rng(11)
    for n in (65, 130, 200):
        sa = "".join(rng.choice(list(LETTERS), n))
        sb = "".join(rng.choice(list(LETTERS), n))
        prod, k = oracle_product_of_strings(oracle, sa, sb)
        ph = 1 + 0j
        for q in range(n):
            m = MATS[sa[q]] @ MATS[sb[q]]
            # find the letter and phase of this qubit's product
            for L in LETTERS:
                for kk in range(4):
                    if np.allclose(m, IK[kk] * MATS[L]):
                        assert prod[q] == L
                        ph *= IK[kk]
        assert np.isclose(ph, IK[k])


# ------------------------------------------------------------------ commutation

def symplectic_inner(sa, sb):
    # Sec. III-F: sum over qubits of x1 z2 XOR z1 x2, mod 2
    s = 0
    for a, b in zip(sa, sb):
        x1, z1 = a in "XY", a in "YZ"
        x2, z2 = b in "XY", b in "YZ"
        s += (x1 and z2) ^ (z1 and x2)
    return s % 2


def test_paper_commutation_examples(oracle):
    for sa, sb, anti in read_golden("paper_commutation.txt"):
        _, k1 = oracle_product_of_strings(oracle, sa, sb)
        _, k2 = oracle_product_of_strings(oracle, sb, sa)
        assert (k1 - k2) % 4 == 2 * int(anti)
        assert symplectic_inner(sa, sb) == int(anti)


def test_phase_parity_is_symplectic_inner_product(oracle):
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 70):
        for _ in range(200):
            sa = "".join(rng.choice(list(LETTERS), n))
            sb = "".join(rng.choice(list(LETTERS), n))
            _, k1 = oracle_product_of_strings(oracle, sa, sb)
            _, k2 = oracle_product_of_strings(oracle, sb, sa)
            w = symplectic_inner(sa, sb)
            assert (k1 - k2) % 4 == 2 * w
            # [P,Q] odd <=> they anti-commute, checked on matrices for small n
            if n <= 5:
                ma, mb = string_matrix(sa), string_matrix(sb)
                assert np.allclose(ma @ mb, (1 - 2 * w) * (mb @ ma))


# ------------------------------------------------------------------ invariants

def test_square_is_identity_and_identity_is_neutral(oracle):
    rng = np.random.default_rng(5)
    for n in (3, 64, 130):
        s = "".join(rng.choice(list(LETTERS), n))
        prod, k = oracle_product_of_strings(oracle, s, s)
        assert prod == "I" * n and k == 0
        prod, k = oracle_product_of_strings(oracle, s, "I" * n)
        assert prod == s and k == 0
        prod, k = oracle_product_of_strings(oracle, "I" * n, s)
        assert prod == s and k == 0


def test_associativity_with_phases(oracle):
    rng = np.random.default_rng(9)
    for n in (4, 66):
        for _ in range(50):
            p, q, r = ("".join(rng.choice(list(LETTERS), n)) for _ in range(3))
            pq, k1 = oracle_product_of_strings(oracle, p, q)
            pqr, k2 = oracle_product_of_strings(oracle, pq, r)
            qr, k3 = oracle_product_of_strings(oracle, q, r)
            pqr2, k4 = oracle_product_of_strings(oracle, p, qr)
            assert pqr == pqr2 and (k1 + k2) % 4 == (k3 + k4) % 4


# ------------------------------------------------------------------ sums

def random_sum(rng, n, m, with_phase=False):
    strs = ["".join(rng.choice(list(LETTERS), n)) for _ in range(m)]
    _, x, z = parse_strings(strs)
    c = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    k = rng.integers(0, 4, m).astype(np.uint8) if with_phase else None
    return strs, x, z, c, k


def sum_matrix(strs, c, k=None):
    M = 0
    for t, s in enumerate(strs):
        ph = IK[int(k[t])] if k is not None else 1
        M = M + ph * c[t] * string_matrix(s)
    return M


@pytest.mark.parametrize("n,ma,mb", [(1, 3, 5), (2, 7, 9), (3, 20, 17), (4, 40, 33)])
def test_canonical_product_equals_matrix_product(oracle, n, ma, mb):
    rng = np.random.default_rng(100 + n)
    sa, ax, az, ac, ak = random_sum(rng, n, ma, with_phase=True)
    sb, bx, bz, bc, bk = random_sum(rng, n, mb, with_phase=True)
    ox, oz, oc, oabs, ocnt = oracle.multiply_canonical(n, (ax, az, ac, ak), (bx, bz, bc, bk))
    out = format_strings(n, ox, oz)
    MA, MB = sum_matrix(sa, ac, ak), sum_matrix(sb, bc, bk)
    M = MA @ MB
    assert np.allclose(sum_matrix(out, oc), M, atol=1e-12, rtol=0)
    # each coefficient is Tr(P M) / 2^n
    for s, c in zip(out, oc):
        assert abs(np.trace(string_matrix(s).conj().T @ M) / 2 ** n - c) < 1e-12
    # key set: every product string occurs, each once, strictly increasing
    keys = keys_as_tuples(ox, oz)
    assert keys == sorted(set(keys))
    expect = {tuple(k) for k in keys_as_tuples(*oracle.multiply_raw(n, (ax, az, ac), (bx, bz, bc))[:2])}
    assert set(keys) == expect
    assert int(ocnt.sum()) == ma * mb


def test_raw_layout_and_phases_vs_kron(oracle):
    rng = np.random.default_rng(42)
    n = 3
    sa, ax, az, ac, ak = random_sum(rng, n, 6, with_phase=True)
    sb, bx, bz, bc, bk = random_sum(rng, n, 5, with_phase=True)
    ox, oz, oc, ok = oracle.multiply_raw(n, (ax, az, ac, ak), (bx, bz, bc, bk))
    out = format_strings(n, ox, oz)
    assert len(out) == 30
    for j in range(5):
        for i in range(6):
            t = j * 6 + i
            lhs = IK[ak[i]] * ac[i] * string_matrix(sa[i]) @ (IK[bk[j]] * bc[j] * string_matrix(sb[j]))
            ar, ai, br, bi = ac[i].real, ac[i].imag, bc[j].real, bc[j].imag
            assert (oc[t].real, oc[t].imag) == (ar * br - ai * bi, ar * bi + ai * br)
            assert np.allclose(lhs, IK[ok[t]] * oc[t] * string_matrix(out[t]))


def test_compress_of_raw_equals_canonical_product(oracle):
    rng = np.random.default_rng(8)
    n = 70
    _, ax, az, ac, _ = random_sum(rng, n, 25)
    # duplicates on purpose: B repeats A's strings
    bx, bz, bc = ax.copy(), az.copy(), rng.standard_normal(25) + 0j
    raw = oracle.multiply_raw(n, (ax, az, ac), (bx, bz, bc))
    c1 = oracle.compress(n, raw)
    c2 = oracle.multiply_canonical(n, (ax, az, ac), (bx, bz, bc))
    for idx in (0, 1, 2, 4):   # keys, coefficients (same summation order), counts
        assert np.array_equal(c1[idx], c2[idx])
    # |c_a c_b| rounded once vs |c_a| |c_b|: equal to a few ulps
    assert np.allclose(c1[3], c2[3], rtol=1e-15, atol=0)


def test_identity_coefficient_closed_form(oracle):
    # For a sum with distinct strings, the identity term of H*H collects c_j^2
    # from P_j P_j = I (Sec. III-A), one contribution per term.
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=16, m=300, seed=5)
    ox, oz, oc, oabs, ocnt = oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())
    ident = [t for t in range(ox.shape[1]) if not ox[:, t].any() and not oz[:, t].any()]
    assert len(ident) == 1
    t = ident[0]
    assert ocnt[t] == h.m
    assert abs(oc[t] - math.fsum((h.c ** 2).real) - 1j * math.fsum((h.c ** 2).imag)) < 1e-15


def test_single_string_product_is_bit_exact_rotation(oracle):
    # A times a single string with coefficient exactly 1: every output
    # coefficient is +-c or +-i c of exactly one input term, bit for bit.
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(1234)
    n = 130
    ax, az = wl.weighted_random(rng, n, 500, 1, n)
    ac = wl.coeffs_loguniform(rng, 500)
    sx, sz = wl.weighted_random(rng, n, 1, 1, n)
    ox, oz, oc, oabs, ocnt = oracle.multiply_canonical(n, (ax, az, ac), (sx, sz, np.ones(1, complex)))
    assert ox.shape[1] == 500 and np.all(ocnt == 1)
    src = {k: t for t, k in enumerate(keys_as_tuples(ax ^ sx, az ^ sz))}
    for u, key in enumerate(keys_as_tuples(ox, oz)):
        re, im = ac[src[key]].real, ac[src[key]].imag
        assert (oc[u].real, oc[u].imag) in ((re, im), (-im, re), (-re, -im), (im, -re))


def test_query_coefficients_match_canonical(oracle):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=20, m=120, seed=77)
    ox, oz, oc, oabs, ocnt = oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())
    qc, qabs, qcnt = oracle.query_product_coeffs(h.n, h.as_tuple(), h.as_tuple(), ox, oz)
    assert np.array_equal(qcnt, ocnt)
    assert np.allclose(qabs, oabs, rtol=1e-14, atol=0)
    assert np.all(np.abs(qc - oc) <= 1e-15 * oabs)
    # a string that is not a product has coefficient 0 and no contributions
    nx = np.zeros_like(ox[:, :1]); nz = np.zeros_like(oz[:, :1])
    nx[0, 0] = 1  # X on qubit 0 alone: odd X-weight, while every JW product has even X-weight
    qc2, _, qcnt2 = oracle.query_product_coeffs(h.n, h.as_tuple(), h.as_tuple(), nx, nz)
    assert qcnt2[0] == 0 and qc2[0] == 0


def test_canonical_order_is_library_sort_of_key_tuples(oracle):
    from paper_2605_25974_gb300 import workloads as wl
    a, b = wl.tiny(n=70, m=40)
    ox, oz, *_ = oracle.multiply_canonical(70, a.as_tuple(), b.as_tuple())
    keys = keys_as_tuples(ox, oz)
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    assert len(keys) == 1600  # random 70-qubit strings: no repeated products


def test_compensated_sum_vs_correctly_rounded_sum(oracle):
    rng = np.random.default_rng(1)
    for _ in range(20):
        v = rng.standard_normal(1000) * 10.0 ** rng.integers(-8, 17, 1000)
        v = np.concatenate([v, -v[:500]])
        rng.shuffle(v)
        exact = math.fsum(v)
        # Neumaier's bound: u|S| + O(n^2 u^2) sum|v|
        bound = 2.0 ** -52 * abs(exact) + 4 * (v.size * 2.0 ** -53) ** 2 * np.abs(v).sum()
        assert abs(oracle.compensated_sum(v) - exact) <= bound
        naive = 0.0
        for t in v:
            naive += t
    assert oracle.compensated_sum(np.array([1e16, 1.0, -1e16])) == 1.0


def _sample_bounds(n, a, b, nsamp, nranges, seed):
    """Sorted distinct keys of sampled product pairs (numpy XOR of the words),
    spaced to cut the key space into about ``nranges`` ranges."""
    rng = np.random.default_rng(seed)
    ia = rng.integers(0, a.m, nsamp)
    jb = rng.integers(0, b.m, nsamp)
    k = np.concatenate([a.x[:, ia] ^ b.x[:, jb], a.z[:, ia] ^ b.z[:, jb]], axis=0).T
    k = np.unique(k, axis=0)  # lexicographic rows, word 0 first
    step = max(1, len(k) // nranges)
    return [k[q] for q in range(step, len(k), step)]


@pytest.mark.parametrize("n,ma,mb,threads", [(20, 200, 150, 3), (130, 120, 90, 4), (64, 300, 1, 2), (5, 40, 40, 5)])
def test_range_mode_concatenates_to_plain_mode(oracle, n, ma, mb, threads):
    # The key-range, threaded canonical product (used for full-size checks)
    # against the plain ordered-map mode: consecutive ranges concatenated give
    # the same keys, counts and |contribution| sums, and coefficients equal up
    # to compensated-summation rounding.
    from paper_2605_25974_gb300 import workloads as wl
    rng = wl.rng_for(900 + n)
    ax, az = wl.weighted_random(rng, n, ma, 1, min(n, 12))
    bx, bz = wl.weighted_random(rng, n, mb, 1, min(n, 12))
    a = wl.SumArrays(n, ax, az, wl.coeffs_normal(rng, ma), rng.integers(0, 4, ma).astype(np.uint8))
    b = wl.SumArrays(n, bx, bz, wl.coeffs_normal(rng, mb), rng.integers(0, 4, mb).astype(np.uint8))
    full = oracle.multiply_canonical(n, a.as_tuple(), b.as_tuple())
    bounds = _sample_bounds(n, a, b, 2000, 6, n)
    edges = [None] + bounds + [None]
    parts = [oracle.multiply_canonical_range(n, a.as_tuple(), b.as_tuple(), lo, hi, threads)
             for lo, hi in zip(edges[:-1], edges[1:])]
    cat = [np.concatenate([p[q] for p in parts], axis=-1) for q in range(5)]
    assert np.array_equal(cat[0], full[0]) and np.array_equal(cat[1], full[1])
    assert np.array_equal(cat[4], full[4])
    assert np.allclose(cat[3], full[3], rtol=1e-15, atol=0)
    err = np.maximum(np.abs(cat[2].real - full[2].real), np.abs(cat[2].imag - full[2].imag))
    assert np.all(err <= 1e-15 * full[3])
    # an empty range and a single-key range
    k0 = np.concatenate([full[0][:, 0], full[1][:, 0]])
    e = oracle.multiply_canonical_range(n, a.as_tuple(), b.as_tuple(), k0, k0, threads)
    assert e[0].shape[1] == 0
    k1 = np.concatenate([full[0][:, 1], full[1][:, 1]])
    one = oracle.multiply_canonical_range(n, a.as_tuple(), b.as_tuple(), k0, k1, threads)
    assert one[0].shape[1] == 1 and one[4][0] == full[4][0]


def test_range_mode_jw_hh_heavy_identity(oracle):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=40, m=300, seed=11)
    full = oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())
    bounds = _sample_bounds(h.n, h, h, 5000, 9, 3)
    edges = [None] + bounds + [None]
    parts = [oracle.multiply_canonical_range(h.n, h.as_tuple(), h.as_tuple(), lo, hi, 4)
             for lo, hi in zip(edges[:-1], edges[1:])]
    x = np.concatenate([p[0] for p in parts], axis=1)
    cnt = np.concatenate([p[4] for p in parts])
    c = np.concatenate([p[2] for p in parts])
    assert np.array_equal(x, full[0]) and np.array_equal(cnt, full[4]) and cnt.max() == 300
    assert np.all(np.abs(c - full[2]) <= 1e-15 * full[3])
