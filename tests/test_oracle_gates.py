"""Pins the oracle's Clifford conjugation and Pauli rotation (Sec. III-B) to
matrices built here with numpy: U Q U^dagger of the full 2^n x 2^n matrices,
decomposed back into Pauli strings by traces, plus the special angles the
paper states (theta = pi flips the sign of anti-commuting terms, theta = pi/2
maps Q to -iPQ) and truncation as a filter of the untruncated result.
"""
import itertools

import numpy as np
import pytest

from conftest import LETTERS, keys_as_tuples, parse_strings, format_strings

MATS = {
    "I": np.array([[1, 0], [0, 1]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
}


def string_matrix(s):
    m = np.array([[1]], dtype=complex)
    for ch in s:  # qubit 0 is the first Kronecker factor
        m = np.kron(m, MATS[ch])
    return m


def gate_full(n, gate, q1, q2):
    """The gate as a 2^n matrix, built from its action on basis states (qubit
    0 is the most significant bit of the basis index)."""
    d = 2 ** n
    U = np.zeros((d, d), complex)
    bit = lambda b, q: (b >> (n - 1 - q)) & 1
    for b in range(d):
        if gate == "h":
            b0 = b & ~(1 << (n - 1 - q1))
            b1 = b | (1 << (n - 1 - q1))
            s = 1 / np.sqrt(2)
            U[b0, b] += s
            U[b1, b] += -s if bit(b, q1) else s
        elif gate == "s":
            U[b, b] = 1j if bit(b, q1) else 1
        elif gate == "cnot":
            U[b ^ (bit(b, q1) << (n - 1 - q2)), b] = 1
        elif gate == "cz":
            U[b, b] = -1 if bit(b, q1) and bit(b, q2) else 1
    return U


def decompose(M, n):
    """Pauli coefficients of M: {string: Tr(P M) / 2^n} for nonzero ones."""
    out = {}
    for letters in itertools.product(LETTERS, repeat=n):
        s = "".join(letters)
        c = np.trace(string_matrix(s).conj().T @ M) / 2 ** n
        if abs(c) > 1e-12:
            out[s] = c
    return out


def random_sum(rng, n, m):
    strs = sorted(set("".join(rng.choice(list(LETTERS), n)) for _ in range(m)))
    _, x, z = parse_strings(strs)
    c = rng.standard_normal(len(strs)) + 1j * rng.standard_normal(len(strs))
    return strs, x, z, c


def sum_matrix(strs, c):
    return sum(ci * string_matrix(s) for s, ci in zip(strs, c))


@pytest.mark.parametrize("gate,q1,q2", [("h", 0, 0), ("h", 2, 0), ("s", 1, 0), ("cnot", 0, 2), ("cnot", 2, 1),
                                        ("cz", 0, 1), ("cz", 2, 0)])
def test_clifford_conjugation_vs_matrices(oracle, gate, q1, q2):
    n = 3
    rng = np.random.default_rng(7)
    strs = ["".join(p) for p in itertools.product(LETTERS, repeat=n)]  # every string once
    _, x, z = parse_strings(strs)
    c = rng.standard_normal(len(strs)) + 1j * rng.standard_normal(len(strs))
    ox, oz, oc = oracle.apply_clifford(n, (x, z, c), gate, q1, q2)
    U = gate_full(n, gate, q1, q2)
    for t, s in enumerate(strs):  # term by term, in order
        img = decompose(U @ string_matrix(s) @ U.conj().T, n)
        assert len(img) == 1  # a Clifford maps a Pauli string to one Pauli string
        (s2, sign), = img.items()
        assert abs(abs(sign) - 1) < 1e-12
        assert format_strings(n, ox[:, t:t + 1], oz[:, t:t + 1])[0] == s2
        assert abs(oc[t] - sign * c[t]) < 1e-12


def test_clifford_known_images(oracle):
    # H: X <-> Z, Y -> -Y; S: X -> Y, Y -> -X; CNOT(0->1): XI -> XX, IZ -> ZZ
    cases = [("h", 0, 0, "X", "Z", 1), ("h", 0, 0, "Y", "Y", -1), ("s", 0, 0, "X", "Y", 1), ("s", 0, 0, "Y", "X", -1),
             ("cnot", 0, 1, "XI", "XX", 1), ("cnot", 0, 1, "IZ", "ZZ", 1), ("cz", 0, 1, "XI", "XZ", 1)]
    for gate, q1, q2, s, s2, sign in cases:
        n, x, z = parse_strings([s])
        ox, oz, oc = oracle.apply_clifford(n, (x, z, np.array([1 + 0j])), gate, q1, q2)
        assert format_strings(n, ox, oz)[0] == s2 and abs(oc[0] - sign) < 1e-12


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.1, np.pi / 2, np.pi, -2.5])
@pytest.mark.parametrize("p", ["XIZ", "YYI", "IZI", "ZXY"])
def test_rotation_vs_matrices(oracle, theta, p):
    n = 3
    rng = np.random.default_rng(int(1000 * theta) % 997 + len(p))
    strs, x, z, c = random_sum(rng, n, 24)
    _, px, pz = parse_strings([p])
    ox, oz, oc, oabs, ocnt = oracle.rotate(n, (x, z, c), px[:, 0], pz[:, 0], theta)
    P = string_matrix(p)
    U = np.cos(theta / 2) * np.eye(2 ** n) - 1j * np.sin(theta / 2) * P
    expect = decompose(U @ sum_matrix(strs, c) @ U.conj().T, n)
    got = dict(zip(format_strings(n, ox, oz), oc))
    assert keys_as_tuples(ox, oz) == sorted(keys_as_tuples(ox, oz))  # canonical order
    for s, v in expect.items():
        assert abs(got.get(s, 0) - v) < 1e-12, (s, got.get(s), v)
    for s, v in got.items():
        assert abs(expect.get(s, 0) - v) < 1e-12, (s, v)


def test_rotation_special_angles(oracle):
    # theta = pi: anti-commuting terms flip sign; theta = pi/2: Q -> -iPQ
    n, x, z = parse_strings(["XI", "ZI", "YZ", "IZ"])
    c = np.array([1.0, 2.0, 3.0j, 4.0 - 1j])
    _, px, pz = parse_strings(["ZI"])
    ox, oz, oc, _, _ = oracle.rotate(n, (x, z, c), px[:, 0], pz[:, 0], np.pi)
    got = dict(zip(format_strings(n, ox, oz), oc))
    assert abs(got["ZI"] - 2.0) < 1e-15 and abs(got["IZ"] - (4.0 - 1j)) < 1e-15
    assert abs(got["XI"] + 1.0) < 1e-15 and abs(got["YZ"] + 3.0j) < 1e-15
    ox, oz, oc, _, _ = oracle.rotate(n, (x, z, c), px[:, 0], pz[:, 0], np.pi / 2)
    got = {s: v for s, v in zip(format_strings(n, ox, oz), oc) if abs(v) > 1e-12}
    # -i Z X = -i (iY) = Y ; -i Z Y = -i (-iX) = -X
    assert abs(got["YI"] - 1.0) < 1e-15 and abs(got["XZ"] + 3.0j) < 1e-15
    assert set(got) == {"YI", "XZ", "ZI", "IZ"}


def test_rotation_truncation_filters_merged_terms(oracle):
    rng = np.random.default_rng(3)
    n = 6
    strs, x, z, c = random_sum(rng, n, 300)
    c = c * np.exp(rng.uniform(-12, 0, len(c)))  # magnitudes over many decades
    _, px, pz = parse_strings(["XYZIXZ"])
    full = oracle.rotate(n, (x, z, c), px[:, 0], pz[:, 0], 0.37)
    tau = 1e-3
    cut = oracle.rotate(n, (x, z, c), px[:, 0], pz[:, 0], 0.37, threshold=tau)
    keep = np.abs(full[2]) >= tau
    assert keep.any() and not keep.all()
    assert np.array_equal(cut[0], full[0][:, keep]) and np.array_equal(cut[1], full[1][:, keep])
    assert np.array_equal(cut[2], full[2][keep])


def test_pairwise_products_vs_kron(oracle):
    # element-wise products against Kronecker matrices, phases of both inputs included
    rng = np.random.default_rng(21)
    n, m = 3, 60
    sa = ["".join(rng.choice(list(LETTERS), n)) for _ in range(m)]
    sb = ["".join(rng.choice(list(LETTERS), n)) for _ in range(m)]
    _, ax, az = parse_strings(sa)
    _, bx, bz = parse_strings(sb)
    ac = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    bc = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    ka = rng.integers(0, 4, m).astype(np.uint8)
    kb = rng.integers(0, 4, m).astype(np.uint8)
    ox, oz, oc, ok = oracle.multiply_pairwise(n, (ax, az, ac, ka), (bx, bz, bc, kb))
    out = format_strings(n, ox, oz)
    ik = np.array([1, 1j, -1, -1j])
    for t in range(m):
        lhs = ac[t] * ik[ka[t]] * string_matrix(sa[t]) @ (bc[t] * ik[kb[t]] * string_matrix(sb[t]))
        rhs = oc[t] * ik[ok[t]] * string_matrix(out[t])
        assert np.allclose(lhs, rhs, atol=1e-12, rtol=0)


def _apply(oracle, n, s, gates):
    x, z, c = s
    for gate, q1, q2 in gates:
        x, z, c = oracle.apply_clifford(n, (x, z, c), gate, q1, q2)
    return x, z, c


def test_clifford_gate_orders(oracle):
    # H^2 = S^4 = CNOT^2 = CZ^2 = identity under conjugation; S^2 (= Z up to a
    # phase) flips the sign of X and Y on its qubit and keeps I and Z
    rng = np.random.default_rng(17)
    n = 4
    strs = ["".join(rng.choice(list(LETTERS), n)) for _ in range(80)]
    _, x, z = parse_strings(strs)
    c = rng.standard_normal(len(strs)) + 1j * rng.standard_normal(len(strs))
    for gates in ([("h", 1, 0)] * 2, [("s", 2, 0)] * 4, [("cnot", 0, 3)] * 2, [("cz", 3, 1)] * 2):
        ox, oz, oc = _apply(oracle, n, (x, z, c), gates)
        assert np.array_equal(ox, x) and np.array_equal(oz, z) and np.array_equal(oc, c)
    ox, oz, oc = _apply(oracle, n, (x, z, c), [("s", 2, 0)] * 2)
    assert np.array_equal(ox, x) and np.array_equal(oz, z)
    flip = np.array([s[2] in "XY" for s in strs])
    assert np.array_equal(oc, np.where(flip, -c, c))


def test_rotations_compose_additively(oracle):
    # U_P(t2) U_P(t1) = U_P(t1 + t2): two steps equal one step by the sum of
    # the angles; a rotation by -t undoes one by t
    rng = np.random.default_rng(23)
    n = 5
    strs = sorted(set("".join(rng.choice(list(LETTERS), n)) for _ in range(60)))
    _, x, z = parse_strings(strs)
    c = rng.standard_normal(len(strs)) + 1j * rng.standard_normal(len(strs))
    _, px, pz = parse_strings(["XZIYZ"])
    px, pz = px[:, 0], pz[:, 0]
    t1, t2 = 0.37, -1.21
    a = oracle.rotate(n, (x, z, c), px, pz, t1)
    b = oracle.rotate(n, (a[0], a[1], a[2]), px, pz, t2)
    one = oracle.rotate(n, (x, z, c), px, pz, t1 + t2)
    got = dict(zip(format_strings(n, b[0], b[1]), b[2]))
    want = dict(zip(format_strings(n, one[0], one[1]), one[2]))
    for s_ in set(got) | set(want):
        assert abs(got.get(s_, 0) - want.get(s_, 0)) < 1e-12
    back = oracle.rotate(n, (a[0], a[1], a[2]), px, pz, -t1)
    got = {s_: v for s_, v in zip(format_strings(n, back[0], back[1]), back[2]) if abs(v) > 1e-12}
    assert got.keys() == set(strs)
    for s_, v in zip(strs, c):
        assert abs(got[s_] - v) < 1e-12


def test_pairwise_products_associative_and_involutive(oracle):
    # (a b) c = a (b c) with phases, and P P = I with phase 0
    rng = np.random.default_rng(29)
    n, m = 70, 40
    sets = [["".join(rng.choice(list(LETTERS), n)) for _ in range(m)] for _ in range(3)]
    (_, ax, az), (_, bx, bz), (_, cx, cz) = [parse_strings(s) for s in sets]
    one = np.ones(m, np.complex128)
    ab = oracle.multiply_pairwise(n, (ax, az, one), (bx, bz, one))
    ab_c = oracle.multiply_pairwise(n, (ab[0], ab[1], one, ab[3]), (cx, cz, one))
    bc = oracle.multiply_pairwise(n, (bx, bz, one), (cx, cz, one))
    a_bc = oracle.multiply_pairwise(n, (ax, az, one), (bc[0], bc[1], one, bc[3]))
    assert np.array_equal(ab_c[0], a_bc[0]) and np.array_equal(ab_c[1], a_bc[1])
    assert np.array_equal(ab_c[3], a_bc[3])
    sq = oracle.multiply_pairwise(n, (ax, az, one), (ax, az, one))
    assert not sq[0].any() and not sq[1].any() and not sq[3].any()
