"""The throughput probes behind the measured rooflines give plausible,
ordered values on the GPU (not a parity test: the oracle has no
counterpart)."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_ordered():
    import paper_1511_01157_gb300 as m
    ctx = m.Context(0)
    try:
        p = ctx.measure_peaks()
    finally:
        ctx.close()
    assert all(v > 0 for v in p.values()), p
    # FP32 FMA issue far above FP64; L1-resident gathers above L2-resident
    assert p["fp32_fma_per_s"] > 4 * p["fp64_fma_per_s"]
    assert p["l1_gather_bytes_per_s"] > p["l2_gather_bytes_per_s"]
    # at most the nominal FP32 issue rate of 152 SMs x 128 lanes x 2.2 GHz
    assert p["fp32_fma_per_s"] < 152 * 128 * 2.2e9 * 1.01
