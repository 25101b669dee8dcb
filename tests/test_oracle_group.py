"""Pins the oracle's greedy commutation grouping (Sec. V-D, the sequential
variant of Sec. IV-C) to facts fixed outside it:

  * commutation decided by the full 2^n x 2^n matrices (PQ == QP), built here
    with numpy Kronecker products;
  * the three properties that define a first-fit partition, checked term by
    term (and which determine it uniquely, by induction over the terms):
    groups are opened in order, a term commutes with every earlier member of
    its group, and every earlier group holds an earlier member that
    anti-commutes with it;
  * the same partition from a different procedure: greedy colouring of the
    anti-commutation graph (each term takes the smallest colour not used by an
    earlier anti-commuting term);
  * closed forms: diagonal strings form one group, the 2n Jordan-Wigner
    Majorana strings anti-commute pairwise and form 2n groups, the paper's
    worked commutation examples (Sec. III-A, tests/golden).
"""
import itertools

import numpy as np
import pytest

from conftest import LETTERS, parse_strings, read_golden

MATS = {
    "I": np.array([[1, 0], [0, 1]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
}


def string_matrix(s):
    m = np.array([[1]], dtype=complex)
    for ch in s:
        m = np.kron(m, MATS[ch])
    return m


def anti_by_matrices(strs):
    """anti[s, t] = 1 when the matrices of strings s and t anti-commute."""
    mats = [string_matrix(s) for s in strs]
    m = len(strs)
    anti = np.zeros((m, m), bool)
    for a in range(m):
        for b in range(a + 1, m):
            pq = mats[a] @ mats[b]
            qp = mats[b] @ mats[a]
            if np.allclose(pq, qp):
                continue
            assert np.allclose(pq, -qp)  # Pauli strings either commute or anti-commute
            anti[a, b] = anti[b, a] = True
    return anti


def check_first_fit(group, ng, anti):
    m = len(group)
    assert ng == (int(group.max()) + 1 if m else 0)
    top = -1
    for t in range(m):
        g = int(group[t])
        assert g <= top + 1, "groups are opened in order"
        top = max(top, g)
        earlier = np.arange(t)
        same = earlier[group[:t] == g]
        assert not anti[same, t].any(), "term %d anti-commutes with a member of its group" % t
        for h in range(g):
            members = earlier[group[:t] == h]
            assert anti[members, t].any(), "term %d fits the earlier group %d" % (t, h)


def greedy_colouring(anti):
    m = anti.shape[0]
    colour = np.zeros(m, np.int32)
    for t in range(m):
        used = set(int(colour[s]) for s in range(t) if anti[s, t])
        c = 0
        while c in used:
            c += 1
        colour[t] = c
    return colour


@pytest.mark.parametrize("n,m,seed", [(1, 12, 1), (2, 40, 2), (3, 150, 3), (4, 120, 4)])
def test_grouping_first_fit_vs_matrices(oracle, n, m, seed):
    rng = np.random.default_rng(seed)
    strs = ["".join(rng.choice(list(LETTERS), n)) for _ in range(m)]  # repeats included
    _, x, z = parse_strings(strs)
    group, ng = oracle.group_commuting(n, x, z)
    anti = anti_by_matrices(strs)
    check_first_fit(group, ng, anti)
    assert np.array_equal(group, greedy_colouring(anti))


def test_grouping_every_string_once(oracle):
    # all 64 strings on 3 qubits, in a shuffled order
    rng = np.random.default_rng(9)
    strs = ["".join(p) for p in itertools.product(LETTERS, repeat=3)]
    strs = [strs[i] for i in rng.permutation(len(strs))]
    _, x, z = parse_strings(strs)
    group, ng = oracle.group_commuting(3, x, z)
    anti = anti_by_matrices(strs)
    check_first_fit(group, ng, anti)
    assert np.array_equal(group, greedy_colouring(anti))


def test_grouping_closed_forms(oracle):
    # one qubit: X, Y, Z pairwise anti-commute; repeats join their own letter's group
    n, x, z = parse_strings(list("XYZXYZI"))
    group, ng = oracle.group_commuting(n, x, z)
    assert group.tolist() == [0, 1, 2, 0, 1, 2, 0] and ng == 3
    # diagonal strings (I and Z only) all commute: one group
    rng = np.random.default_rng(5)
    strs = ["".join(rng.choice(list("IZ"), 500)) for _ in range(64)]
    n, x, z = parse_strings(strs)
    group, ng = oracle.group_commuting(n, x, z)
    assert ng == 1 and not group.any()
    # the 2n Majorana strings Z..Z X I..I and Z..Z Y I..I anti-commute pairwise
    q = 40
    maj = []
    for k in range(q):
        for ch in "XY":
            maj.append("Z" * k + ch + "I" * (q - k - 1))
    n, x, z = parse_strings(maj)
    group, ng = oracle.group_commuting(n, x, z)
    assert group.tolist() == list(range(2 * q)) and ng == 2 * q
    # the identity commutes with everything: first Majorana joins its group
    n, x, z = parse_strings(["I" * q] + maj)
    group, ng = oracle.group_commuting(n, x, z)
    assert group.tolist() == [0, 0] + list(range(1, 2 * q)) and ng == 2 * q


def test_grouping_paper_commutation_examples(oracle):
    for sa, sb, anti in read_golden("paper_commutation.txt"):
        n, x, z = parse_strings([sa, sb])
        group, ng = oracle.group_commuting(n, x, z)
        assert group.tolist() == ([0, 1] if int(anti) else [0, 0])


def test_grouping_empty(oracle):
    group, ng = oracle.group_commuting(5, np.zeros((1, 0), np.uint64), np.zeros((1, 0), np.uint64))
    assert ng == 0 and group.shape == (0,)


def test_grouping_500_qubits_first_fit(oracle):
    # the paper's grouping workload shape at a small size; commutation from the
    # letters (Sec. III-A), computed with numpy, independent of the oracle's C
    from paper_2605_25974_gb300 import workloads as wl
    from paper_2605_25974_gb300.workloads import unpack_bits
    h = wl.grouping(300)
    group, ng = oracle.group_commuting(h.n, h.x, h.z)
    xb = unpack_bits(h.x, h.n)
    zb = unpack_bits(h.z, h.n)
    letter = xb.astype(np.int8) + 2 * zb.astype(np.int8)  # 0 = I, any nonzero = a Pauli letter
    nz = letter != 0
    diff = (letter[:, None, :] != letter[None, :, :]) & nz[:, None, :] & nz[None, :, :]
    anti = (diff.sum(-1) % 2).astype(bool)
    check_first_fit(group, ng, anti)
    assert 1 < ng < 300
