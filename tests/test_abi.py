"""The C-ABI library builds for sm_103a and exports every symbol the public
header declares.  No compute call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "paulib.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(paulib_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_25974_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_expected_entry_points():
    from paper_2605_25974_gb300 import paulib
    assert set(header_symbols()) == set(paulib.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_abi_version(lib):
    lib.paulib_abi_version.restype = ctypes.c_int32
    assert lib.paulib_abi_version() == 3


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2605_25974_gb300 import paulib
    saved = paulib._lib
    paulib._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            paulib.load(str(tmp_path / "missing.so"))
    finally:
        paulib._lib = saved


def test_invalid_arguments_rejected_without_gpu(lib):
    # argument checks happen before any device call
    lib.paulib_sum_create.restype = ctypes.c_int32
    lib.paulib_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    st = lib.paulib_sum_create(0, 1, None, None, None, None, None, ctypes.byref(out))
    assert st == 1 and out.value is None
    assert b"n_qubits" in lib.paulib_last_error()
    st = lib.paulib_sum_create(2000, 1, None, None, None, None, None, ctypes.byref(out))
    assert st == 1
    st = lib.paulib_sum_create(10, -1, None, None, None, None, None, ctypes.byref(out))
    assert st == 1


def test_gate_rotation_grouping_arguments_rejected_without_gpu(lib):
    # the NEXT-row entry points check their arguments before any device call
    lib.paulib_last_error.restype = ctypes.c_char_p
    for name in ("paulib_apply_clifford", "paulib_rotate", "paulib_multiply_pairwise", "paulib_group_commuting",
                 "paulib_set_group_candidates"):
        getattr(lib, name).restype = ctypes.c_int32
    ng = ctypes.c_int64(-1)
    assert lib.paulib_group_commuting(None, None, None, None, ctypes.byref(ng), None) == 1
    assert lib.paulib_apply_clifford(None, 0, None, None) == 1
    out = ctypes.c_void_p()
    assert lib.paulib_rotate(None, None, None, ctypes.c_double(0.1), ctypes.c_double(0.0), 0, None,
                             ctypes.byref(out)) == 1
    assert lib.paulib_multiply_pairwise(None, None, None, ctypes.byref(out)) == 1
    # grouping tuning: 1..4 candidates per term
    assert lib.paulib_set_group_candidates(0) == 1 and b"1..4" in lib.paulib_last_error()
    assert lib.paulib_set_group_candidates(5) == 1
    assert lib.paulib_set_group_candidates(2) == 0
    assert lib.paulib_set_group_candidates(4) == 0
