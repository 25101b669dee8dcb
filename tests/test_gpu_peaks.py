"""paulib_measure_peaks: the pipe rates the roofline divides by must be
positive and of the order a GB300 can deliver (wide bounds; the exact values
are measurements, reported by the benchmark)."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_plausible():
    import torch
    from paper_2605_25974_gb300 import paulib
    from paper_2605_25974_gb300.build import build
    build()
    torch.cuda.init()
    p = paulib.measure_peaks()
    assert set(p) == set(paulib.PEAK_NAMES)
    assert 1e10 < p["fp64_fma_per_s"] < 1e14
    assert 1e12 < p["fp32_fma_per_s"] < 1e15
    assert 1e12 < p["lop3_per_s"] < 1e15
    assert 1e12 < p["iadd_per_s"] < 1e15
    assert 1e11 < p["popc_per_s"] < 1e15
    assert 1e11 < p["l2_gather64_bytes_per_s"] < 1e14
    assert 1e11 < p["l2_gather32_bytes_per_s"] < 1e14
