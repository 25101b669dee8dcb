"""Greedy commutation grouping (Sec. V-D) on the GPU against the CPU oracle,
through the C ABI.  The group of every term and the number of groups must be
identical (integer work: bit-exact); the CSR listing must be the partition
written out in term order.  Sizes span one 64-term block, ragged blocks, every
availability-row width the kernel has (held in shared or global memory), and
the degenerate cases: empty and one-term sums, all strings commuting (one
group), all anti-commuting (one group per term), repeated strings."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2605_25974_gb300 import paulib
    from paper_2605_25974_gb300.build import build
    build()
    torch.cuda.init()
    return paulib


def run(lib, s, csr=True):
    with lib.PauliSum.from_arrays(s) as g:
        grp, ng, off, mem = lib.group_commuting(g, csr=csr)
        import torch
        torch.cuda.synchronize()
        return (grp.cpu().numpy(), ng, None if off is None else off.cpu().numpy(),
                None if mem is None else mem.cpu().numpy())


def check_csr(grp, ng, off, mem):
    counts = np.bincount(grp, minlength=ng)
    assert off.shape == (ng + 1,) and off[0] == 0
    assert np.array_equal(np.diff(off), counts)
    order = np.lexsort((np.arange(len(grp)), grp))  # by group, then term
    assert np.array_equal(mem, order)


def sum_of(strs_x, strs_z, n):
    from paper_2605_25974_gb300 import workloads as wl
    m = strs_x.shape[1]
    return wl.SumArrays(n, strs_x, strs_z, np.ones(m, np.complex128))


@pytest.mark.parametrize("m", [1, 2, 63, 64, 65, 200, 1000, 2000, 2500])
def test_grouping_random_500_qubits(lib, oracle, m):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.grouping(m)
    grp, ng, off, mem = run(lib, h)
    og, ong = oracle.group_commuting(h.n, h.x, h.z)
    assert ng == ong
    assert np.array_equal(grp, og)
    check_csr(grp, ng, off, mem)


@pytest.mark.parametrize("n,m", [(64, 5000), (64, 10000), (20, 3000), (130, 4100), (1024, 700)])
def test_grouping_row_widths(lib, oracle, n, m):
    # 5000 and 4100 terms: rows of 4 words per lane in shared memory; 10000:
    # 8 words per lane with the group masks in global memory
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.grouping(m, n=n, seed=7 * n + m)
    grp, ng, off, mem = run(lib, h)
    og, ong = oracle.group_commuting(h.n, h.x, h.z)
    assert ng == ong and np.array_equal(grp, og)
    check_csr(grp, ng, off, mem)


def test_grouping_jordan_wigner(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.jw(n=100, m=3000, seed=77)
    grp, ng, off, mem = run(lib, h)
    og, ong = oracle.group_commuting(h.n, h.x, h.z)
    assert ng == ong and np.array_equal(grp, og)
    check_csr(grp, ng, off, mem)


def test_grouping_majoranas_repeated(lib, oracle):
    # the 2n Majorana strings anti-commute pairwise: one group each; a second
    # and third copy of the list (and the identity) join the first copy's groups
    from conftest import parse_strings
    q = 500
    maj = []
    for k in range(q):
        for ch in "XY":
            maj.append("Z" * k + ch + "I" * (q - k - 1))
    strs = ["I" * q] + maj + maj[::-1] + maj
    n, x, z = parse_strings(strs)
    grp, ng, off, mem = run(lib, sum_of(x, z, n))
    og, ong = oracle.group_commuting(n, x, z)
    assert ng == ong == 2 * q and np.array_equal(grp, og)
    check_csr(grp, ng, off, mem)


def test_grouping_all_commuting_and_empty(lib, oracle):
    rng = np.random.default_rng(3)
    from paper_2605_25974_gb300.workloads import pack_bits
    n, m = 300, 3000
    zb = rng.integers(0, 2, (m, n)).astype(bool)
    x = pack_bits(np.zeros((m, n), bool), n)
    z = pack_bits(zb, n)
    grp, ng, off, mem = run(lib, sum_of(x, z, n))
    assert ng == 1 and not grp.any()
    check_csr(grp, ng, off, mem)
    # empty sum: no groups, offsets [0]
    with lib.PauliSum.create(n, np.zeros((5, 0), np.uint64), np.zeros((5, 0), np.uint64),
                             np.zeros(0, np.complex128)) as g:
        grp, ng, off, mem = lib.group_commuting(g)
        assert ng == 0 and grp.numel() == 0 and off.cpu().tolist() == [0]


def test_grouping_without_csr_and_repeats(lib, oracle):
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.grouping(700, n=9, seed=5)  # 9 qubits: many repeated and commuting strings
    idx = np.random.default_rng(1).integers(0, h.m, 1500)
    r = h.subset(idx)
    grp, ng, off, mem = run(lib, r, csr=False)
    og, ong = oracle.group_commuting(r.n, r.x, r.z)
    assert off is None and mem is None
    assert ng == ong and np.array_equal(grp, og)


def test_grouping_errors(lib):
    import ctypes
    L = lib.load()
    ng = ctypes.c_int64(0)
    assert L.paulib_group_commuting(None, None, None, None, ctypes.byref(ng), None) == 1
    from paper_2605_25974_gb300 import workloads as wl
    with lib.PauliSum.from_arrays(wl.grouping(10)) as g:
        assert L.paulib_group_commuting(ctypes.c_void_p(g.handle), None, None, None, ctypes.byref(ng), None) == 1


def test_grouping_40000_terms_properties(lib):
    # 40,000 terms on 64 qubits: rows of 16 words per lane, everything in
    # global memory.  Too large for the oracle; checked by the properties that
    # define the first-fit partition on sampled terms, with commutation from
    # the symplectic parity of the words
    from paper_2605_25974_gb300 import workloads as wl
    h = wl.grouping(40000, n=64, seed=40000)
    grp, ng, off, mem = run(lib, h)
    check_csr(grp, ng, off, mem)
    assert grp[0] == 0 and np.all(grp[1:] <= np.maximum.accumulate(grp)[:-1] + 1)
    x, z = h.x[0], h.z[0]
    rng = np.random.default_rng(2)
    for t in rng.choice(h.m, 60, replace=False):
        s = np.arange(t)
        w = (x[t] & z[s]) ^ (z[t] & x[s])
        anti = np.array([bin(int(v)).count("1") & 1 for v in w], bool)
        g = grp[t]
        assert not anti[grp[s] == g].any()
        blocked = np.zeros(ng, bool)
        blocked[grp[s][anti]] = True
        assert blocked[:g].all()


@pytest.mark.parametrize("k", [1, 2])
def test_grouping_row_scan_path(lib, oracle, k):
    # keeping fewer candidates per term sends many terms to the whole-row scan
    # (taken candidates cleared from the term's row); the partition is the same
    from paper_2605_25974_gb300 import workloads as wl
    try:
        lib.set_group_candidates(k)
        for m, n, seed in [(3000, 500, 11), (2500, 64, 12), (1200, 9, 13)]:
            h = wl.grouping(m, n=n, seed=seed)
            grp, ng, off, mem = run(lib, h)
            og, ong = oracle.group_commuting(h.n, h.x, h.z)
            assert ng == ong and np.array_equal(grp, og), (m, n, k)
            check_csr(grp, ng, off, mem)
    finally:
        lib.set_group_candidates(4)
    with pytest.raises(lib.PaulibError):
        lib.set_group_candidates(0)
