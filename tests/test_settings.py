"""Argument checks of the library's settings, which are host state only: the
canonicalisation tuning, the slot sort, the persistent batched kernel's sizes
and the test knobs reject out-of-range values with INVALID_ARG and accept
the documented ones.  No compute call is made (no GPU needed); each test
restores the defaults it changed."""
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2605_25974_gb300 import paulib
    from paper_2605_25974_gb300.build import build
    build()
    paulib.load()
    return paulib


def test_batch_tuning_ranges(lib):
    for ok in ((0, 0), (32, 1), (2048, 8), (-1, -1), (512, 3)):
        lib.set_batch_tuning(*ok)
    for bad in ((31, 2), (4096, 2), (0, 9), (-2, 0), (16, -2)):
        with pytest.raises(lib.PaulibError, match="INVALID_ARG"):
            lib.set_batch_tuning(*bad)
    lib.set_batch_tuning(0, 0)


def test_slot_tuning_ranges(lib):
    lib.set_slot_tuning(0, 0, 1024, 120, 8)
    lib.set_slot_tuning(0, 1, 0, 0, 0)
    for bad in ((0, 2, -1, -1, -1), (0, -1, 8, -1, -1), (0, -1, 5000, -1, -1), (0, -1, -1, -1, 65),
                (0, -1, -1, -2, -1)):
        with pytest.raises(lib.PaulibError, match="INVALID_ARG"):
            lib.set_slot_tuning(*bad)


def test_debug_knob_ranges(lib):
    for knob, value in ((1, 3), (1, 0), (2, 16), (2, 0), (3, 1), (3, 0), (4, 32), (4, 2048), (4, 0)):
        lib.set_debug(knob, value)
    for knob, value in ((0, 1), (5, 1), (1, 65), (1, -1), (2, 5000), (3, 2), (4, 31), (4, 4096)):
        with pytest.raises(lib.PaulibError, match="INVALID_ARG"):
            lib.set_debug(knob, value)
