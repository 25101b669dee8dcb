"""Seeded synthetic Pauli-sum generators shared by the tests, the benchmark and
the oracle checks.

This module only draws random inputs and packs bits; it contains none of the
Pauli-product or canonicalisation arithmetic, so neither side of a parity
check can borrow the other's logic through it.

Layout of every generated sum (the paper's struct-of-arrays form, Sec. IV-A):
``x`` and ``z`` are uint64 arrays of shape (W, M) with W = ceil(n/64), qubit q
at word q//64, bit q%64 (Table I: I=(0,0), Z=(0,1), X=(1,0), Y=(1,1)); ``c`` is
complex128 of shape (M,).  Every generated sum has distinct strings, except
the batched workload's (see ``batch``).

Workloads (the paper's benchmarks use unnamed random sums, Sec. VI; the
chemistry-shaped one stands in for Jordan-Wigner molecular Hamiltonians,
Sec. III-A, Eq. 2):

* ``tiny``: two 64-term sums at n=20, every qubit uniform over {I,X,Y,Z},
  re/im ~ N(0,1); seeds 101 and 102.
* ``stream``: a 1,000,000-term sum at n=500, weight uniform in [1,500] on
  distinct random qubits with letters uniform over {X,Y,Z}, |c| log-uniform
  on [1e-6,1] with uniform phase (seed 201), times 256 single strings of the
  same distribution with coefficient exactly 1 (seed 202).
* ``jw``: Jordan-Wigner-shaped Hamiltonians: n single-Z terms, 10% ZZ pairs,
  20% one-body hops (X/Y at p<q joined by a Z run), the rest two-body terms
  (X/Y at p<q<r<s with Z runs inside (p,q) and (r,s)); |c| log-uniform on
  [1e-6,1], uniform phase.  n=100/M=20,000 (seed 301) and n=200/M=30,000
  (seed 401); H*H is the product.
* ``grouping``: random n=500 sums for greedy commutation grouping (the
  paper's grouping benchmark, Sec. VI-C, uses random 500-qubit sums of 200 to
  2,000 terms): every qubit uniform over {I,X,Y,Z}, distinct strings,
  re/im ~ N(0,1); seed 600 + M // 100 for M terms.
* ``batch``: 4,096 independent products at n=500; left sizes
  floor(exp(U(ln 16, ln 16384))), right sizes uniform in 1..8, strings of
  weight at most 32 on random qubits (repeats allowed), coefficients as in
  ``stream``; one stream of seed 501, vectorised over problems.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np


@dataclasses.dataclass
class SumArrays:
    """A Pauli sum as plain host arrays (SoA words + complex coefficients)."""
    n: int
    x: np.ndarray                 # (W, M) uint64
    z: np.ndarray                 # (W, M) uint64
    c: np.ndarray                 # (M,) complex128
    k: Optional[np.ndarray] = None  # (M,) uint8 phase exponents, or None (= all 0)

    @property
    def m(self) -> int:
        return int(self.x.shape[1])

    @property
    def words(self) -> int:
        return int(self.x.shape[0])

    def as_tuple(self):
        if self.k is None:
            return (self.x, self.z, self.c)
        return (self.x, self.z, self.c, self.k)

    def subset(self, idx) -> "SumArrays":
        return SumArrays(self.n, np.ascontiguousarray(self.x[:, idx]), np.ascontiguousarray(self.z[:, idx]),
                         np.ascontiguousarray(self.c[idx]), None if self.k is None else self.k[idx])


def words_for(n: int) -> int:
    return (n + 63) // 64


def rng_for(seed: int, sub: Optional[int] = None) -> np.random.Generator:
    if sub is None:
        return np.random.Generator(np.random.PCG64(seed))
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=(sub,))))


def pack_bits(bits: np.ndarray, n: int) -> np.ndarray:
    """(M, n) bool -> (W, M) uint64, qubit q at word q//64 bit q%64."""
    m = bits.shape[0]
    W = words_for(n)
    pad = np.zeros((m, W * 64), dtype=bool)
    pad[:, :n] = bits
    by = np.packbits(pad, axis=1, bitorder="little")          # (M, 8W) bytes, byte b = bits 8b..8b+7
    words = by.view("<u8").reshape(m, W)
    return np.ascontiguousarray(words.T.astype(np.uint64))


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    """(W, M) uint64 -> (M, n) bool (inverse of :func:`pack_bits`)."""
    W, m = words.shape
    by = np.ascontiguousarray(words.T.astype("<u8")).view(np.uint8).reshape(m, W * 8)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :n].astype(bool)


def _letters_to_bits(letters: np.ndarray):
    """letters 0=I,1=X,2=Y,3=Z -> (xbits, zbits) per Table I."""
    xb = (letters == 1) | (letters == 2)
    zb = (letters == 3) | (letters == 2)
    return xb, zb


def _dedupe(x: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Indices of the first occurrence of each distinct (x, z) column."""
    key = np.concatenate([x, z], axis=0).T                    # (M, 2W)
    key = np.ascontiguousarray(key).view(np.dtype((np.void, key.dtype.itemsize * key.shape[1]))).ravel()
    _, first = np.unique(key, return_index=True)
    return np.sort(first)


def _topup(draw, m: int):
    """Draws rows with ``draw(count) -> (x, z)`` until m distinct strings exist."""
    xs, zs = draw(m)
    keep = _dedupe(xs, zs)
    xs, zs = xs[:, keep], zs[:, keep]
    while xs.shape[1] < m:
        need = m - xs.shape[1]
        nx, nz = draw(max(16, int(need * 1.25)))
        xs = np.concatenate([xs, nx], axis=1)
        zs = np.concatenate([zs, nz], axis=1)
        keep = _dedupe(xs, zs)
        xs, zs = xs[:, keep], zs[:, keep]
    return np.ascontiguousarray(xs[:, :m]), np.ascontiguousarray(zs[:, :m])


def coeffs_normal(rng: np.random.Generator, m: int) -> np.ndarray:
    return (rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex128)


def coeffs_loguniform(rng: np.random.Generator, m: int, lo: float = 1e-6, hi: float = 1.0) -> np.ndarray:
    mag = 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=m)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=m)
    return (mag * np.cos(ph) + 1j * mag * np.sin(ph)).astype(np.complex128)


# ---------------------------------------------------------------- string families

def uniform_letters(rng: np.random.Generator, n: int, m: int):
    """Every qubit uniform over {I, X, Y, Z}."""
    def draw(cnt):
        L = rng.integers(0, 4, size=(cnt, n))
        xb, zb = _letters_to_bits(L)
        return pack_bits(xb, n), pack_bits(zb, n)
    return _topup(draw, m)


def weighted_random(rng: np.random.Generator, n: int, m: int, wmin: int, wmax: int, chunk: int = 65536):
    """Weight uniform in [wmin, wmax] on distinct random qubits, letters uniform {X, Y, Z}."""
    def draw(cnt):
        xs, zs = [], []
        for s in range(0, cnt, chunk):
            r = min(chunk, cnt - s)
            w = rng.integers(wmin, wmax + 1, size=r)
            if wmax * 8 <= n:
                pos, valid = _small_subsets(rng, n, r, w)
            else:
                perm = rng.permuted(np.tile(np.arange(n, dtype=np.int32), (r, 1)), axis=1)
                pos = perm
                valid = np.arange(n)[None, :] < w[:, None]
            letters = rng.integers(1, 4, size=pos.shape)
            L = np.zeros((r, n), dtype=np.int8)
            rows = np.broadcast_to(np.arange(r)[:, None], pos.shape)
            L[rows[valid], pos[valid]] = letters[valid]
            xb, zb = _letters_to_bits(L)
            xs.append(pack_bits(xb, n))
            zs.append(pack_bits(zb, n))
        return np.concatenate(xs, axis=1), np.concatenate(zs, axis=1)
    return _topup(draw, m)


def _small_subsets(rng, n, r, w):
    """For each row a uniformly random w[row]-subset of range(n) (w small):
    sequential draws with duplicates rejected, in draw order."""
    wmax = int(w.max()) if w.size else 0
    draws = max(2 * wmax, wmax + 16)
    while True:
        vals = rng.integers(0, n, size=(r, draws))
        order = np.argsort(vals, axis=1, kind="stable")
        sv = np.take_along_axis(vals, order, axis=1)
        dup_sorted = np.zeros_like(sv, dtype=bool)
        dup_sorted[:, 1:] = sv[:, 1:] == sv[:, :-1]
        dup = np.zeros_like(dup_sorted)
        np.put_along_axis(dup, order, dup_sorted, axis=1)
        fresh = ~dup
        rank = np.cumsum(fresh, axis=1)
        if np.all(rank[:, -1] >= w):
            valid = fresh & (rank <= w[:, None])
            return vals, valid
        draws *= 2


def jw_hamiltonian(rng: np.random.Generator, n: int, m: int):
    """Jordan-Wigner-shaped string set (see module docstring); m distinct strings."""
    n_z = n
    n_zz = int(round(0.10 * m))
    n_1b = int(round(0.20 * m))
    n_2b = m - n_z - n_zz - n_1b
    if n_2b < 0:
        raise ValueError("m too small for n")
    parts_x, parts_z = [], []

    # single-Z terms on every qubit
    L = np.zeros((n_z, n), dtype=np.int8)
    L[np.arange(n), np.arange(n)] = 3
    xb, zb = _letters_to_bits(L)
    parts_x.append(pack_bits(xb, n)); parts_z.append(pack_bits(zb, n))

    def sorted_positions(cnt, k):
        p = np.sort(rng.random((cnt, n)).argsort(axis=1)[:, :k], axis=1) if cnt * n <= 4_000_000 else None
        if p is None:
            v, valid = _small_subsets(rng, n, cnt, np.full(cnt, k))
            p = np.sort(v[valid].reshape(cnt, k), axis=1)
        return p

    def draw_zz(cnt):
        p = sorted_positions(cnt, 2)
        L = np.zeros((cnt, n), dtype=np.int8)
        L[np.arange(cnt), p[:, 0]] = 3
        L[np.arange(cnt), p[:, 1]] = 3
        xb, zb = _letters_to_bits(L)
        return pack_bits(xb, n), pack_bits(zb, n)

    idx = np.arange(n)[None, :]

    def draw_1b(cnt):
        p = sorted_positions(cnt, 2)
        L = np.zeros((cnt, n), dtype=np.int8)
        run = (idx > p[:, :1]) & (idx < p[:, 1:2])
        L[run] = 3
        xy = rng.integers(1, 3, size=(cnt, 2))
        L[np.arange(cnt), p[:, 0]] = xy[:, 0]
        L[np.arange(cnt), p[:, 1]] = xy[:, 1]
        xb, zb = _letters_to_bits(L)
        return pack_bits(xb, n), pack_bits(zb, n)

    def draw_2b(cnt):
        p = sorted_positions(cnt, 4)
        L = np.zeros((cnt, n), dtype=np.int8)
        run = ((idx > p[:, :1]) & (idx < p[:, 1:2])) | ((idx > p[:, 2:3]) & (idx < p[:, 3:4]))
        L[run] = 3
        xy = rng.integers(1, 3, size=(cnt, 4))
        for c in range(4):
            L[np.arange(cnt), p[:, c]] = xy[:, c]
        xb, zb = _letters_to_bits(L)
        return pack_bits(xb, n), pack_bits(zb, n)

    for cnt, fn in ((n_zz, draw_zz), (n_1b, draw_1b), (n_2b, draw_2b)):
        if cnt > 0:
            x, z = _topup(fn, cnt)
            parts_x.append(x); parts_z.append(z)
    return np.concatenate(parts_x, axis=1), np.concatenate(parts_z, axis=1)


# ---------------------------------------------------------------- named workloads

def tiny(seed_a: int = 101, seed_b: int = 102, n: int = 20, m: int = 64) -> Tuple[SumArrays, SumArrays]:
    out = []
    for s in (seed_a, seed_b):
        rng = rng_for(s)
        x, z = uniform_letters(rng, n, m)
        out.append(SumArrays(n, x, z, coeffs_normal(rng, m)))
    return out[0], out[1]


def stream(m: int = 1_000_000, strings: int = 256, n: int = 500, seed_a: int = 201, seed_b: int = 202):
    ra = rng_for(seed_a)
    x, z = weighted_random(ra, n, m, 1, n)
    a = SumArrays(n, x, z, coeffs_loguniform(ra, m))
    rb = rng_for(seed_b)
    bx, bz = weighted_random(rb, n, strings, 1, n)
    singles = [SumArrays(n, bx[:, s:s + 1].copy(), bz[:, s:s + 1].copy(), np.ones(1, np.complex128))
               for s in range(strings)]
    return a, singles


def jw(n: int = 100, m: int = 20_000, seed: int = 301) -> SumArrays:
    rng = rng_for(seed)
    x, z = jw_hamiltonian(rng, n, m)
    return SumArrays(n, x, z, coeffs_loguniform(rng, m))


def grouping(m: int = 2000, n: int = 500, seed: Optional[int] = None) -> SumArrays:
    rng = rng_for(600 + m // 100 if seed is None else seed)
    x, z = uniform_letters(rng, n, m)
    return SumArrays(n, x, z, coeffs_normal(rng, m))


def low_weight_terms(rng: np.random.Generator, n: int, m: int, wmax: int, chunk: int = 1 << 20):
    """m strings with at most wmax non-identity qubits: a weight w uniform in
    1..wmax, then w qubit positions and letters uniform over {X, Y, Z}; a
    position drawn twice keeps its first letter, so the weight is at most w.
    Strings may repeat; canonicalisation merges them."""
    W = words_for(n)
    xo = np.zeros((W, m), np.uint64)
    zo = np.zeros((W, m), np.uint64)
    for s0 in range(0, m, chunk):
        r = min(chunk, m - s0)
        w = rng.integers(1, wmax + 1, size=r)
        pos = rng.integers(0, n, size=(r, wmax)).astype(np.int32)
        let = rng.integers(1, 4, size=(r, wmax)).astype(np.int8)
        use = np.arange(wmax)[None, :] < w[:, None]
        # sort each row's positions (unused slots last) and keep the first of equal ones
        key = np.where(use, pos, n + 1)
        order = np.argsort(key, axis=1, kind="stable")
        pos = np.take_along_axis(key, order, axis=1)
        let = np.take_along_axis(let, order, axis=1)
        keep = pos < n
        keep[:, 1:] &= pos[:, 1:] != pos[:, :-1]
        # distinct bits of one word add up to their OR; sum 32-bit halves exactly in float64
        rows = np.broadcast_to(np.arange(r, dtype=np.int64)[:, None], pos.shape)[keep]
        p = pos[keep].astype(np.int64)
        lt = let[keep]
        flat = rows * W + p // 64
        b = p % 64
        wgt = np.ldexp(1.0, (b % 32).astype(np.int32))
        lo = b < 32
        for sel, out in (((lt == 1) | (lt == 2), xo), ((lt == 2) | (lt == 3), zo)):
            acc_lo = np.bincount(flat, weights=np.where(sel & lo, wgt, 0.0), minlength=r * W)
            acc_hi = np.bincount(flat, weights=np.where(sel & ~lo, wgt, 0.0), minlength=r * W)
            words = acc_lo.astype(np.uint64) | (acc_hi.astype(np.uint64) << np.uint64(32))
            out[:, s0:s0 + r] = words.reshape(r, W).T
    return xo, zo


def batch(problems: int = 4096, n: int = 500, seed: int = 501, amin: int = 16, amax: int = 16384,
          bmax: int = 8, wmax: int = 32) -> List[Tuple[SumArrays, SumArrays]]:
    """Independent products shaped like Pauli-propagation steps: left sizes
    floor(exp(U(ln amin, ln amax))), right sizes uniform in 1..bmax, strings of
    weight <= wmax, coefficients log-uniform in magnitude with uniform phase.
    All draws come from one stream in a fixed order (sizes, then left terms,
    right terms, left and right coefficients), vectorised over problems."""
    rng = rng_for(seed)
    na = np.floor(np.exp(rng.uniform(math.log(amin), math.log(amax), size=problems))).astype(np.int64)
    nb = rng.integers(1, bmax + 1, size=problems)
    ax, az = low_weight_terms(rng, n, int(na.sum()), wmax)
    bx, bz = low_weight_terms(rng, n, int(nb.sum()), wmax)
    ac = coeffs_loguniform(rng, int(na.sum()))
    bc = coeffs_loguniform(rng, int(nb.sum()))
    oa = np.concatenate([[0], np.cumsum(na)])
    ob = np.concatenate([[0], np.cumsum(nb)])
    out = []
    for q in range(problems):
        sa = slice(int(oa[q]), int(oa[q + 1]))
        sb = slice(int(ob[q]), int(ob[q + 1]))
        out.append((SumArrays(n, np.ascontiguousarray(ax[:, sa]), np.ascontiguousarray(az[:, sa]), ac[sa].copy()),
                    SumArrays(n, np.ascontiguousarray(bx[:, sb]), np.ascontiguousarray(bz[:, sb]), bc[sb].copy())))
    return out


WORKLOADS = {
    "tiny_n20_64x64": "two 64-term sums at n=20, uniform letters, N(0,1) coefficients",
    "stream_n500_1m_x256": "1M-term n=500 sum times 256 single strings",
    "jw_hh_n100_m20000": "H*H, Jordan-Wigner-shaped H at n=100 with 20,000 terms",
    "jw_hh_n200_m30000": "H*H, Jordan-Wigner-shaped H at n=200 with 30,000 terms",
    "batch_n500_4096": "4,096 independent sum x sum products at n=500",
}
