"""Thin ctypes binding over ``libpaulib.so`` (declared in ``include/paulib.h``).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Host arrays are numpy arrays; device arrays are torch
CUDA tensors (PyTorch provides device memory and streams, nothing else).
There is no CPU fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from .build import LIB as _LIB_PATH

OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "QUBIT_MISMATCH", 3: "TAIL_BITS", 4: "OOM", 5: "CUDA",
          6: "TIMEOUT", 7: "UNSUPPORTED", 8: "INTERNAL"}
PRECISION = {"fp64": 0, "fp32_fp64merge": 1, "fp32_twosum": 2}
OUT_RAW, OUT_CANONICAL = 0, 1

# Every symbol include/paulib.h declares.
EXPORTED = ["paulib_abi_version", "paulib_sum_create", "paulib_sum_info", "paulib_sum_export",
            "paulib_sum_destroy", "paulib_multiply", "paulib_compress", "paulib_multiply_batched",
            "paulib_last_error", "paulib_set_allocator", "paulib_timing_enable", "paulib_timing_read",
            "paulib_multiply_noalloc", "paulib_batch_plan_create", "paulib_batch_plan_launch",
            "paulib_batch_plan_outputs", "paulib_batch_plan_destroy", "paulib_set_tuning",
            "paulib_apply_clifford", "paulib_rotate", "paulib_multiply_pairwise",
            "paulib_group_commuting", "paulib_set_group_candidates", "paulib_set_slot_tuning",
            "paulib_last_canon_method", "paulib_sum_export_range", "paulib_last_canon_stats", "paulib_set_debug",
            "paulib_measure_peaks", "paulib_set_batch_tuning"]
GATES = {"h": 0, "s": 1, "cnot": 2, "cz": 3}
STAGES = ["convert", "sample", "count", "scatter", "level2", "compact", "raw", "export", "leaf", "group", "split",
          "place"]


class PaulibError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), msg))
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


def library_path() -> str:
    return _LIB_PATH


def load(path: Optional[str] = None):
    """Opens the library (no build, no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libpaulib.so not found at %s: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)" % p)
    lib = ctypes.CDLL(p)
    lib.paulib_abi_version.restype = _i32
    lib.paulib_sum_create.argtypes = [_i32, _i64, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]
    lib.paulib_sum_info.argtypes = [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64), ctypes.POINTER(_i32)]
    lib.paulib_sum_export.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    lib.paulib_sum_destroy.argtypes = [_vp]
    lib.paulib_sum_destroy.restype = None
    lib.paulib_multiply.argtypes = [_vp, _vp, _i32, _i32, _vp, ctypes.POINTER(_vp)]
    lib.paulib_compress.argtypes = [_vp, _i32, _vp, ctypes.POINTER(_vp)]
    lib.paulib_multiply_batched.argtypes = [_i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, _vp,
                                            ctypes.POINTER(_vp)]
    lib.paulib_last_error.restype = ctypes.c_char_p
    lib.paulib_batch_plan_create.argtypes = [_i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, _vp,
                                             ctypes.POINTER(_vp)]
    lib.paulib_batch_plan_create.restype = _i32
    lib.paulib_batch_plan_launch.argtypes = [_vp, _vp]
    lib.paulib_batch_plan_launch.restype = _i32
    lib.paulib_batch_plan_outputs.argtypes = [_vp, _vp, ctypes.POINTER(_vp)]
    lib.paulib_batch_plan_outputs.restype = _i32
    lib.paulib_batch_plan_destroy.argtypes = [_vp]
    lib.paulib_batch_plan_destroy.restype = None
    lib.paulib_set_tuning.argtypes = [_i32, _i32, _i32, _i32, _i32]
    lib.paulib_set_tuning.restype = _i32
    lib.paulib_timing_enable.argtypes = [_i32]
    lib.paulib_timing_enable.restype = _i32
    lib.paulib_timing_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _i32]
    lib.paulib_timing_read.restype = _i32
    lib.paulib_apply_clifford.argtypes = [_vp, _i32, _vp, _vp]
    lib.paulib_apply_clifford.restype = _i32
    lib.paulib_rotate.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _i32, _vp, ctypes.POINTER(_vp)]
    lib.paulib_rotate.restype = _i32
    lib.paulib_multiply_pairwise.argtypes = [_vp, _vp, _vp, ctypes.POINTER(_vp)]
    lib.paulib_multiply_pairwise.restype = _i32
    lib.paulib_group_commuting.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(_i64), _vp]
    lib.paulib_group_commuting.restype = _i32
    lib.paulib_set_group_candidates.argtypes = [_i32]
    lib.paulib_set_group_candidates.restype = _i32
    lib.paulib_set_batch_tuning.argtypes = [_i32, _i32]
    lib.paulib_set_batch_tuning.restype = _i32
    lib.paulib_set_slot_tuning.argtypes = [_i32, _i32, _i32, _i32, _i32]
    lib.paulib_set_slot_tuning.restype = _i32
    lib.paulib_last_canon_method.argtypes = [ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
    lib.paulib_last_canon_method.restype = _i32
    lib.paulib_sum_export_range.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp]
    lib.paulib_sum_export_range.restype = _i32
    lib.paulib_last_canon_stats.argtypes = [ctypes.POINTER(_i64)]
    lib.paulib_last_canon_stats.restype = _i32
    lib.paulib_set_debug.argtypes = [_i32, _i64]
    lib.paulib_set_debug.restype = _i32
    lib.paulib_measure_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), _i32, _vp]
    lib.paulib_measure_peaks.restype = _i32
    for name in ("paulib_sum_create", "paulib_sum_info", "paulib_sum_export", "paulib_multiply",
                 "paulib_compress", "paulib_multiply_batched", "paulib_set_allocator"):
        getattr(lib, name).restype = _i32
    _lib = lib
    return lib


def _check(st: int):
    if st != OK:
        raise PaulibError(st, load().paulib_last_error().decode(errors="replace"))


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _words(n):
    return (n + 63) // 64


def _prec(p) -> int:
    return PRECISION[p] if isinstance(p, str) else int(p)


class PauliSum:
    """Owning handle of a device-resident sum."""

    def __init__(self, handle: int):
        self._h = handle
        n, m, c = _i32(), _i64(), _i32()
        _check(load().paulib_sum_info(_vp(handle), ctypes.byref(n), ctypes.byref(m), ctypes.byref(c)))
        self.n_qubits, self.n_terms, self.is_canonical = n.value, m.value, bool(c.value)

    @property
    def handle(self) -> int:
        return self._h

    @property
    def words(self) -> int:
        return _words(self.n_qubits)

    @classmethod
    def create(cls, n_qubits: int, x, z, c, k=None, stream=None) -> "PauliSum":
        """x, z: (W, M) uint64; c: (M,) complex128 (or (M, 2) float64); k: (M,) uint8.
        Host (numpy, contiguous) or device (torch CUDA) arrays."""
        m = int(x.shape[-1]) if x.ndim == 2 else int(x.shape[0])
        keep = []
        arrs = []
        for a in (x, z, c, k):
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a)
            keep.append(a)
            arrs.append(_ptr(a))
        out = _vp()
        _check(load().paulib_sum_create(int(n_qubits), int(m), arrs[0], arrs[1], arrs[2], arrs[3],
                                        _vp(_stream(stream)), ctypes.byref(out)))
        return cls(out.value)

    @classmethod
    def from_arrays(cls, s, stream=None) -> "PauliSum":
        """From a ``workloads.SumArrays``."""
        return cls.create(s.n, s.x, s.z, s.c, s.k, stream=stream)

    def export(self, x=None, z=None, c=None, k=None, stream=None, with_phase=True):
        """Copies the sum out (into the given host/device buffers, or new host
        arrays).  Synchronises the stream before returning host arrays."""
        W, m = self.words, self.n_terms
        if x is None:
            x = np.zeros((W, m), np.uint64)
            z = np.zeros((W, m), np.uint64)
            c = np.zeros(m, np.complex128)
            k = np.zeros(m, np.uint8) if with_phase else None
        st = _stream(stream)
        _check(load().paulib_sum_export(_vp(self._h), _ptr(x), _ptr(z), _ptr(c), _ptr(k), _vp(st)))
        if isinstance(x, np.ndarray) or (hasattr(x, "is_cuda") and not x.is_cuda):
            import torch
            if stream is None:
                torch.cuda.current_stream().synchronize()
            elif hasattr(stream, "synchronize"):
                stream.synchronize()
            else:
                torch.cuda.synchronize()
        return x, z, c, k

    def export_range(self, first, count, stream=None, with_phase=False):
        """Copies terms [first, first + count) out into new host arrays."""
        W = self.words
        x = np.zeros((W, count), np.uint64)
        z = np.zeros((W, count), np.uint64)
        c = np.zeros(count, np.complex128)
        k = np.zeros(count, np.uint8) if with_phase else None
        st = _stream(stream)
        _check(load().paulib_sum_export_range(_vp(self._h), ctypes.c_int64(first), ctypes.c_int64(count), _ptr(x),
                                              _ptr(z), _ptr(c), _ptr(k), _vp(st)))
        import torch
        if stream is None:
            torch.cuda.current_stream().synchronize()
        elif hasattr(stream, "synchronize"):
            stream.synchronize()
        else:
            torch.cuda.synchronize()
        return x, z, c, k

    def close(self):
        if self._h:
            load().paulib_sum_destroy(_vp(self._h))
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def multiply(a: PauliSum, b: PauliSum, precision="fp64", canonical: bool = True, stream=None) -> PauliSum:
    out = _vp()
    _check(load().paulib_multiply(_vp(a.handle), _vp(b.handle), _prec(precision),
                                  OUT_CANONICAL if canonical else OUT_RAW, _vp(_stream(stream)),
                                  ctypes.byref(out)))
    return PauliSum(out.value)


def compress(s: PauliSum, precision="fp64", stream=None) -> PauliSum:
    out = _vp()
    _check(load().paulib_compress(_vp(s.handle), _prec(precision), _vp(_stream(stream)), ctypes.byref(out)))
    return PauliSum(out.value)


def multiply_batched(a: Sequence[PauliSum], b: Sequence[PauliSum], precision="fp64",
                     stream=None) -> List[PauliSum]:
    n = len(a)
    A = (_vp * n)(*[s.handle for s in a])
    B = (_vp * n)(*[s.handle for s in b])
    O = (_vp * n)()
    _check(load().paulib_multiply_batched(n, A, B, _prec(precision), _vp(_stream(stream)), O))
    return [PauliSum(O[i]) for i in range(n)]


class _Borrowed(PauliSum):
    """A sum owned by a batch plan: never destroyed through this handle."""

    def close(self):
        self._h = 0


class BatchPlan:
    """Prepared batched product: ``launch`` enqueues it without allocating or
    synchronising (capturable in a CUDA graph); ``outputs`` syncs and returns
    the plan-owned canonical sums of the last launch."""

    def __init__(self, a: Sequence[PauliSum], b: Sequence[PauliSum], precision="fp64", stream=None):
        n = len(a)
        self.batch = n
        self._keep = (list(a), list(b))
        A = (_vp * n)(*[s.handle for s in a])
        B = (_vp * n)(*[s.handle for s in b])
        out = _vp()
        _check(load().paulib_batch_plan_create(n, A, B, _prec(precision), _vp(_stream(stream)), ctypes.byref(out)))
        self._h = out.value

    def launch(self, stream=None):
        _check(load().paulib_batch_plan_launch(_vp(self._h), _vp(_stream(stream))))

    def outputs(self, stream=None) -> List[PauliSum]:
        O = (_vp * self.batch)()
        _check(load().paulib_batch_plan_outputs(_vp(self._h), _vp(_stream(stream)), O))
        return [_Borrowed(O[i]) for i in range(self.batch)]

    def close(self):
        if self._h:
            load().paulib_batch_plan_destroy(_vp(self._h))
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def timing_enable(on: bool = True):
    _check(load().paulib_timing_enable(1 if on else 0))


def timing_read(reset: bool = True):
    """Per-stage device milliseconds and kernel launch counts since the last reset."""
    n = len(STAGES)
    ms = (ctypes.c_double * n)()
    la = (_i64 * n)()
    _check(load().paulib_timing_read(ms, la, 1 if reset else 0))
    return ({s: ms[i] for i, s in enumerate(STAGES)}, {s: int(la[i]) for i, s in enumerate(STAGES)})


def set_tuning(key_words=0, coarse_factor=0, oversample=0, count_ctas_per_sm=0, range_ctas_per_sm=0):
    """Pipeline tuning for keys of ``key_words`` words (0 = all); 0 keeps a value."""
    _check(load().paulib_set_tuning(int(key_words), int(coarse_factor), int(oversample), int(count_ctas_per_sm),
                                    int(range_ctas_per_sm)))


def set_batch_tuning(leaf_cap=-1, split_fan=-1):
    """Sizes of the persistent batched kernel for plans made afterwards:
    leaf capacity (0 = compiled) and split fan-out (0 = 2); -1 keeps a
    value.  Results never depend on them."""
    _check(load().paulib_set_batch_tuning(int(leaf_cap), int(split_fan)))


def set_slot_tuning(key_words=0, method=-1, leaf_cap=-1, slot_target=-1, slot_oversample=-1):
    """Canonicalisation method (0 slot sort, 1 range sort) and slot-sort
    tuning for keys of ``key_words`` words (0 = all): -1 keeps a value, 0
    restores its default."""
    _check(load().paulib_set_slot_tuning(int(key_words), int(method), int(leaf_cap), int(slot_target),
                                         int(slot_oversample)))


def last_canon_method():
    """(method, fallback_bits) of this thread's last canonical result: method 0
    slot sort, 1 range sort; fallback_bits nonzero when the slot sort handed
    the call to the range sort."""
    m, b = _i32(), _i32()
    _check(load().paulib_last_canon_method(ctypes.byref(m), ctypes.byref(b)))
    return int(m.value), int(b.value)


PEAK_NAMES = ("fp64_fma_per_s", "fp32_fma_per_s", "lop3_per_s", "iadd_per_s", "popc_per_s",
              "l2_gather64_bytes_per_s", "l2_gather32_bytes_per_s")


def measure_peaks(stream=None):
    """Measured pipe rates (dict, see paulib_measure_peaks)."""
    v = (ctypes.c_double * len(PEAK_NAMES))()
    _check(load().paulib_measure_peaks(v, len(PEAK_NAMES), _vp(_stream(stream))))
    return dict(zip(PEAK_NAMES, [float(q) for q in v]))


def set_debug(knob, value):
    """Test settings: knob 1 = warp-leaf hash bits kept (forces the hash-clash
    path), knob 2 = range-CTA worklist capacity (forces the stack error),
    knob 3 = 1: batch plans made afterwards take the general pipeline,
    knob 4 = the persistent batched kernel's leaf capacity (forces its
    splits on small inputs); value 0 turns a setting off."""
    _check(load().paulib_set_debug(int(knob), int(value)))


def last_canon_stats():
    """Shape of this thread's last slot sort: ranges, slot capacity per range,
    leaves, leaf capacity, slot target."""
    v = (_i64 * 5)()
    _check(load().paulib_last_canon_stats(v))
    return dict(zip(("ranges", "slots_per_range", "leaves", "leaf_cap", "slot_target"), [int(q) for q in v]))


def apply_clifford(s: "PauliSum", gates, stream=None):
    """Conjugates every term of ``s`` in place by a list of Clifford gates
    [(gate, q1[, q2]), ...], gate in "h", "s", "cnot", "cz" (applied in order)."""
    ops = np.zeros((len(gates), 3), np.int32)
    for g, op in enumerate(gates):
        ops[g, 0] = GATES[op[0]] if isinstance(op[0], str) else int(op[0])
        ops[g, 1] = int(op[1])
        ops[g, 2] = int(op[2]) if len(op) > 2 else 0
    _check(load().paulib_apply_clifford(_vp(s.handle), len(gates), _vp(ops.ctypes.data), _vp(_stream(stream))))
    if len(gates):
        s.is_canonical = False  # relabelled strings are no longer in key order


def rotate(s: "PauliSum", p_x, p_z, theta: float, threshold: float = 0.0, precision="fp64",
           stream=None) -> "PauliSum":
    """Pauli-propagation step under exp(-i theta P / 2): a new canonical sum,
    truncated at |c| < threshold (when threshold > 0).  P is given as
    ceil(n/64) x- and z-words (numpy arrays or device tensors)."""
    W = _words(s.n_qubits)
    if isinstance(p_x, np.ndarray):
        p_x = np.ascontiguousarray(p_x, dtype=np.uint64).reshape(W)
        p_z = np.ascontiguousarray(p_z, dtype=np.uint64).reshape(W)
    out = _vp()
    _check(load().paulib_rotate(_vp(s.handle), _vp(_ptr(p_x)), _vp(_ptr(p_z)), float(theta), float(threshold),
                                _prec(precision), _vp(_stream(stream)), ctypes.byref(out)))
    return PauliSum(out.value)


def multiply_pairwise(a: "PauliSum", b: "PauliSum", stream=None) -> "PauliSum":
    """Element-wise products a_t * b_t as a new raw sum (phases kept)."""
    out = _vp()
    _check(load().paulib_multiply_pairwise(_vp(a.handle), _vp(b.handle), _vp(_stream(stream)), ctypes.byref(out)))
    return PauliSum(out.value)


def group_commuting(s: "PauliSum", csr: bool = True, stream=None):
    """Greedy first-fit partition of the terms into mutually commuting groups
    (terms in order; each joins the first group it commutes with entirely).
    Returns (group of each term, number of groups, offsets, members) as device
    int32 tensors; offsets (G+1,) and members (M,) are None unless csr."""
    import torch
    m = s.n_terms
    # one allocation: group of each term, then the offsets, then the members
    buf = torch.empty(3 * m + 1 if csr else max(m, 1), dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    ng = _i64(0)
    _check(load().paulib_group_commuting(_vp(s.handle), _vp(p), _vp(p + 4 * m if csr else None),
                                         _vp(p + 4 * (2 * m + 1) if csr else None), ctypes.byref(ng),
                                         _vp(_stream(stream))))
    g = int(ng.value)
    if not csr:
        return buf[:m], g, None, None
    group, offsets, members = torch.split(buf, [m, m + 1, m])
    return group, g, offsets[:g + 1], members


def set_group_candidates(k: int):
    """Groups each term keeps at the start of its 64-term block (1..4); the
    partition never depends on it."""
    _check(load().paulib_set_group_candidates(int(k)))
