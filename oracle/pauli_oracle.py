"""ctypes front end of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module.  Every function here forwards to
``paulib_oracle.cpp``, the plain qubit-by-qubit definition of the Pauli-sum
product (PauLIB Sec. III-A), its outer product (Sec. IV-C) and its canonical
sort-and-combine form (Sec. III-H).

Sums are passed as numpy arrays in the paper's struct-of-arrays layout
(Sec. IV-A): ``x``/``z`` of shape (W, M) uint64 with W = ceil(n/64),
``c`` complex128 of shape (M,), optional phase exponents ``k`` uint8 (M,)
meaning the term is i^k c P.
"""
import ctypes
import numpy as np

from .build import build_oracle

_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        lib.oracle_string_product.restype = ctypes.c_int
        lib.oracle_multiply_canonical.restype = ctypes.c_void_p
        lib.oracle_multiply_canonical_range.restype = ctypes.c_void_p
        lib.oracle_compress.restype = ctypes.c_void_p
        lib.oracle_result_size.restype = ctypes.c_int64
        lib.oracle_result_size.argtypes = [ctypes.c_void_p]
        lib.oracle_result_copy.argtypes = [ctypes.c_void_p, _u64p, _u64p, _f64p, _f64p, _i64p]
        lib.oracle_result_free.argtypes = [ctypes.c_void_p]
        lib.oracle_compensated_sum.restype = ctypes.c_double
        lib.oracle_rotate.restype = ctypes.c_void_p
        lib.oracle_group_commuting.restype = ctypes.c_int64
        lib.oracle_group_commuting.argtypes = [ctypes.c_int, ctypes.c_int64, _u64p, _u64p, _i32p]
        lib.oracle_rotate.argtypes = [ctypes.c_int, ctypes.c_int64, _u64p, _u64p, _f64p, _u8p, _u64p, _u64p,
                                      ctypes.c_double, ctypes.c_double]
        _lib = lib
    return _lib


def _p(a, t):
    if a is None:
        return ctypes.cast(None, t)
    return a.ctypes.data_as(t)


def _words(n):
    return (n + 63) // 64


def _prep(n, x, z, c, k):
    W = _words(n)
    x = np.ascontiguousarray(x, dtype=np.uint64).reshape(W, -1)
    z = np.ascontiguousarray(z, dtype=np.uint64).reshape(W, -1)
    m = x.shape[1]
    cc = np.ascontiguousarray(np.asarray(c, dtype=np.complex128).reshape(m)).view(np.float64)
    kk = None if k is None else np.ascontiguousarray(k, dtype=np.uint8).reshape(m)
    return x, z, cc, kk, m


def letter_product(a, b):
    """Single-qubit product of letters (0=I, 1=X, 2=Y, 3=Z): (letter, k)."""
    lib = _load()
    ol, ok = ctypes.c_int(), ctypes.c_int()
    lib.oracle_letter_product(int(a), int(b), ctypes.byref(ol), ctypes.byref(ok))
    return ol.value, ok.value


def string_product(n, xa, za, xb, zb):
    """Product of two strings given as W-word arrays: (x, z, k)."""
    lib = _load()
    W = _words(n)
    xa, za, xb, zb = (np.ascontiguousarray(v, dtype=np.uint64).reshape(W) for v in (xa, za, xb, zb))
    xo = np.zeros(W, np.uint64)
    zo = np.zeros(W, np.uint64)
    k = lib.oracle_string_product(int(n), _p(xa, _u64p), _p(za, _u64p), _p(xb, _u64p), _p(zb, _u64p),
                                  _p(xo, _u64p), _p(zo, _u64p))
    return xo, zo, k


def multiply_raw(n, a, b):
    """Raw outer product; ``a``/``b`` are (x, z, c[, k]) tuples.

    Returns (x, z, c, k) with |A|*|B| terms, slot j*|A| + i = a_i * b_j.
    """
    lib = _load()
    ax, az, ac, ak, na = _prep(n, *a[:3], a[3] if len(a) > 3 else None)
    bx, bz, bc, bk, nb = _prep(n, *b[:3], b[3] if len(b) > 3 else None)
    W = _words(n)
    nout = na * nb
    ox = np.zeros((W, nout), np.uint64)
    oz = np.zeros((W, nout), np.uint64)
    oc = np.zeros(nout, np.complex128)
    ok = np.zeros(nout, np.uint8)
    lib.oracle_multiply_raw(int(n), ctypes.c_int64(na), _p(ax, _u64p), _p(az, _u64p), _p(ac, _f64p),
                            _p(ak, _u8p), ctypes.c_int64(nb), _p(bx, _u64p), _p(bz, _u64p),
                            _p(bc, _f64p), _p(bk, _u8p), _p(ox, _u64p), _p(oz, _u64p),
                            _p(oc.view(np.float64), _f64p), _p(ok, _u8p))
    return ox, oz, oc, ok


def _take(h, W):
    lib = _load()
    u = lib.oracle_result_size(h)
    ox = np.zeros((W, u), np.uint64)
    oz = np.zeros((W, u), np.uint64)
    oc = np.zeros(u, np.complex128)
    oabs = np.zeros(u, np.float64)
    ocnt = np.zeros(u, np.int64)
    lib.oracle_result_copy(h, _p(ox, _u64p), _p(oz, _u64p), _p(oc.view(np.float64), _f64p),
                           _p(oabs, _f64p), _p(ocnt, _i64p))
    lib.oracle_result_free(h)
    return ox, oz, oc, oabs, ocnt


def multiply_canonical(n, a, b):
    """Canonical product A*B: (x, z, c, abs_sum, count), ascending key order."""
    lib = _load()
    ax, az, ac, ak, na = _prep(n, *a[:3], a[3] if len(a) > 3 else None)
    bx, bz, bc, bk, nb = _prep(n, *b[:3], b[3] if len(b) > 3 else None)
    h = lib.oracle_multiply_canonical(int(n), ctypes.c_int64(na), _p(ax, _u64p), _p(az, _u64p),
                                      _p(ac, _f64p), _p(ak, _u8p), ctypes.c_int64(nb), _p(bx, _u64p),
                                      _p(bz, _u64p), _p(bc, _f64p), _p(bk, _u8p))
    return _take(ctypes.c_void_p(h), _words(n))


def multiply_canonical_range(n, a, b, lo=None, hi=None, threads=1):
    """Terms of the canonical product A*B whose key lies in [lo, hi), computed
    with ``threads`` host threads.  lo/hi are 2W-word keys (x words then z
    words) or None for an open end.  Returns (x, z, c, abs_sum, count) as
    multiply_canonical does; consecutive ranges concatenate to the whole sum."""
    lib = _load()
    ax, az, ac, ak, na = _prep(n, *a[:3], a[3] if len(a) > 3 else None)
    bx, bz, bc, bk, nb = _prep(n, *b[:3], b[3] if len(b) > 3 else None)
    W = _words(n)
    lo_a = None if lo is None else np.ascontiguousarray(np.asarray(lo, dtype=np.uint64).reshape(2 * W))
    hi_a = None if hi is None else np.ascontiguousarray(np.asarray(hi, dtype=np.uint64).reshape(2 * W))
    h = lib.oracle_multiply_canonical_range(int(n), ctypes.c_int64(na), _p(ax, _u64p), _p(az, _u64p),
                                            _p(ac, _f64p), _p(ak, _u8p), ctypes.c_int64(nb), _p(bx, _u64p),
                                            _p(bz, _u64p), _p(bc, _f64p), _p(bk, _u8p), _p(lo_a, _u64p),
                                            _p(hi_a, _u64p), int(threads))
    return _take(ctypes.c_void_p(h), W)


def compress(n, s):
    """Canonical form of one sum ``s`` = (x, z, c[, k])."""
    lib = _load()
    x, z, c, k, m = _prep(n, *s[:3], s[3] if len(s) > 3 else None)
    h = lib.oracle_compress(int(n), ctypes.c_int64(m), _p(x, _u64p), _p(z, _u64p), _p(c, _f64p),
                            _p(k, _u8p))
    return _take(ctypes.c_void_p(h), _words(n))


def query_product_coeffs(n, a, b, qx, qz):
    """Coefficient of each query string in A*B from the definition.

    Returns (coef complex128, abs_sum, count) per query.
    """
    lib = _load()
    ax, az, ac, ak, na = _prep(n, *a[:3], a[3] if len(a) > 3 else None)
    bx, bz, bc, bk, nb = _prep(n, *b[:3], b[3] if len(b) > 3 else None)
    W = _words(n)
    qx = np.ascontiguousarray(qx, dtype=np.uint64).reshape(W, -1)
    qz = np.ascontiguousarray(qz, dtype=np.uint64).reshape(W, -1)
    nq = qx.shape[1]
    oc = np.zeros(nq, np.complex128)
    oabs = np.zeros(nq, np.float64)
    ocnt = np.zeros(nq, np.int64)
    lib.oracle_query_product_coeffs(int(n), ctypes.c_int64(na), _p(ax, _u64p), _p(az, _u64p),
                                    _p(ac, _f64p), _p(ak, _u8p), ctypes.c_int64(nb), _p(bx, _u64p),
                                    _p(bz, _u64p), _p(bc, _f64p), _p(bk, _u8p), ctypes.c_int64(nq),
                                    _p(qx, _u64p), _p(qz, _u64p), _p(oc.view(np.float64), _f64p),
                                    _p(oabs, _f64p), _p(ocnt, _i64p))
    return oc, oabs, ocnt


def compensated_sum(v):
    lib = _load()
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib.oracle_compensated_sum(ctypes.c_int64(v.size), _p(v, _f64p))


GATES = {"h": 0, "s": 1, "cnot": 2, "cz": 3}


def apply_clifford(n, s, gate, q1, q2=0):
    """Conjugation U Q U^dagger of every term of ``s`` = (x, z, c[, k]) by a
    Clifford gate ("h", "s", "cnot" with control q1 and target q2, "cz"), from
    the gate's matrix (Sec. III-B).  Terms keep their order; returns
    (x, z, c) with the input phase and the image's sign folded into c."""
    lib = _load()
    x, z, c, k, m = _prep(n, *s[:3], s[3] if len(s) > 3 else None)
    W = _words(n)
    ox = np.zeros((W, m), np.uint64)
    oz = np.zeros((W, m), np.uint64)
    oc = np.zeros(m, np.complex128)
    lib.oracle_apply_clifford(int(n), ctypes.c_int64(m), _p(x, _u64p), _p(z, _u64p), _p(c, _f64p), _p(k, _u8p),
                              int(GATES[gate]), int(q1), int(q2), _p(ox, _u64p), _p(oz, _u64p),
                              _p(oc.view(np.float64), _f64p))
    return ox, oz, oc


def rotate(n, s, px, pz, theta, threshold=0.0):
    """Conjugation of every term by U_P(theta) = exp(-i theta P / 2), merged
    into canonical form, then truncated at |c| < threshold (when > 0):
    (x, z, c, abs_sum, count)."""
    lib = _load()
    x, z, c, k, m = _prep(n, *s[:3], s[3] if len(s) > 3 else None)
    W = _words(n)
    px = np.ascontiguousarray(px, dtype=np.uint64).reshape(W)
    pz = np.ascontiguousarray(pz, dtype=np.uint64).reshape(W)
    h = lib.oracle_rotate(int(n), ctypes.c_int64(m), _p(x, _u64p), _p(z, _u64p), _p(c, _f64p), _p(k, _u8p),
                          _p(px, _u64p), _p(pz, _u64p), float(theta), float(threshold))
    return _take(ctypes.c_void_p(h), W)


def multiply_pairwise(n, a, b):
    """Element-wise products a_t * b_t of equally long term lists: (x, z, c, k)."""
    lib = _load()
    ax, az, ac, ak, m = _prep(n, *a[:3], a[3] if len(a) > 3 else None)
    bx, bz, bc, bk, mb = _prep(n, *b[:3], b[3] if len(b) > 3 else None)
    assert m == mb
    W = _words(n)
    ox = np.zeros((W, m), np.uint64)
    oz = np.zeros((W, m), np.uint64)
    oc = np.zeros(m, np.complex128)
    ok = np.zeros(m, np.uint8)
    lib.oracle_multiply_pairwise(int(n), ctypes.c_int64(m), _p(ax, _u64p), _p(az, _u64p), _p(ac, _f64p), _p(ak, _u8p),
                                 _p(bx, _u64p), _p(bz, _u64p), _p(bc, _f64p), _p(bk, _u8p), _p(ox, _u64p),
                                 _p(oz, _u64p), _p(oc.view(np.float64), _f64p), _p(ok, _u8p))
    return ox, oz, oc, ok


def group_commuting(n, x, z):
    """Greedy first-fit commutation grouping of the strings (x, z) in their
    order: (group index of each term as int32 (M,), number of groups)."""
    lib = _load()
    W = _words(n)
    x = np.ascontiguousarray(x, dtype=np.uint64).reshape(W, -1)
    z = np.ascontiguousarray(z, dtype=np.uint64).reshape(W, -1)
    m = x.shape[1]
    grp = np.zeros(m, np.int32)
    ng = lib.oracle_group_commuting(int(n), ctypes.c_int64(m), _p(x, _u64p), _p(z, _u64p), _p(grp, _i32p))
    return grp, int(ng)
