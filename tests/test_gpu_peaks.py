"""The roofline denominators the benchmark measures itself (hrr_measure_peaks): each is
positive and within a broad physical range for one GB300-class GPU, and the scattered
record fetch is slower than the streaming read it is compared with."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    import paper_1907_12343_gb300 as hrr
    ctx = hrr.Context(0)
    p = ctx.measure_peaks()
    ctx.close()
    assert 1e3 < p["l2_read_gbs"] < 1e5
    assert 1e9 < p["record_fetches_per_s"] < 1e12
    assert 1e12 < p["int_ops_per_s"] < 1e14
    # 64 bytes per scattered record at most reach the streaming rate
    assert 64.0 * p["record_fetches_per_s"] / 1e9 < 1.5 * p["l2_read_gbs"]
