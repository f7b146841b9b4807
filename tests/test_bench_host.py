"""Host logic of the benchmark (no GPU): the source keys that decide whether a committed
DRAM profile still describes the kernel, the profile lookup, the roofline fractions, and
the workload description both arms share."""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def test_code_key_ignores_comments_and_whitespace_only(bench):
    code = "int f(int a) {\n  return a + 1; // add\n}\n/* block\n comment */\n"
    same = "int f(int a) { return a + 1; }  // other words\n"
    other = "int f(int a) { return a + 2; }\n"
    assert bench._code_only(code) == bench._code_only(same)
    assert bench._code_only(code) != bench._code_only(other)


def test_profile_applies_only_to_its_workload_and_shape(bench):
    # the committed summary names its workload and hierarchy shape; any other one gets no
    # traffic figure, whatever the sources
    assert bench.profiled_traffic("480x270x1048576") is None
    assert bench.profiled_traffic("1920x1080x1048576", topology="radix") is None
    t = bench.profiled_traffic("1920x1080x1048576", topology="cost")
    assert t is None or t > 1e9  # present exactly when the kernel and build code are unchanged


def test_fractions_arithmetic(bench):
    measured = {"l2_read_gbs": 20000.0, "record_fetches_per_s": 1e11, "int_ops_per_s": 4e13}
    peaks = {"hbm_gbs": 6000.0}
    f = bench.other_fractions(V=1e9, accepted=1e6, n_e=1000, n_l=1001, sec=0.01, peaks=peaks,
                              measured=measured, tile_bytes=16384)
    assert f["record_fetch"]["frac"] == pytest.approx(1e11 / 1e11)
    assert f["l2_stream"]["achieved_gbs"] == pytest.approx(64e9 / 0.01 / 1e9)
    unique = 64.0 * 1000 + 16.0 * 1000 + 16384 + 8.0 * 1e6
    assert f["hbm"]["unique_bytes"] == pytest.approx(unique)
    assert f["int32"]["achieved_per_s"] == pytest.approx(1e9 * bench.OPS_PER_VISIT / 0.01)
    assert bench.other_fractions(1, 1, 1, 2, 1.0, {}, {}, 0) == {}


def test_both_arms_describe_the_same_workload(bench):
    args = argparse.Namespace(eyes="1920x1080")
    a = bench.frame_config(args, 2073600, 1048576, 3e-6, 30, 1)
    assert a["topology"] == bench.TOPOLOGY and a["n_eyes"] == 2073600 and a["parallelism"] == "replicas x1"
    assert set(a) >= {"workload", "n_eyes", "n_lights", "tau", "tree_height", "step", "topology", "l2"}


def test_l2_figures_come_from_the_small_frame_profile(bench):
    l2 = bench.profiled_l2()
    assert l2 is None or (l2["workload"] == "480x270x1048576" and l2["l2_bytes_per_s"] > 1e12
                          and 0 < l2["l2_throughput_pct"] <= 100)
    assert bench.profiled_l2(topology="radix") is None
