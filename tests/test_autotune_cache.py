"""Host logic of the per-size-class autotuner: class keys, the JSON cache, and that a class
is tuned once (on a bounded sample) and reused after. A fake context stands in for the
library, so no GPU is needed."""
import json

import numpy as np
import pytest

from paper_1907_12343_gb300.autotune import Autotuner, size_class

torch = pytest.importorskip("torch")


class FakeCtx:
    def __init__(self):
        self.calls = []

    def autotune_all(self, x, y, z, px, py, tree, tau, pairs):
        self.calls.append(int(x.numel()))
        best = {"rangemin_variant": 2, "blocks_per_sm": 5, "node_width": 4, "ring_entries": 256,
                "threads_per_block": 128}
        other = dict(best, node_width=2, blocks_per_sm=6)
        return [(other, 1.5), (best, 1.25), (dict(best, rangemin_variant=0), 1.3)]


def _eyes(n):
    z = torch.zeros(n)
    return z, z, z, torch.zeros(n, dtype=torch.int16), torch.zeros(n, dtype=torch.int16)


def test_size_class_groups_by_bit_length():
    assert size_class(1920 * 1080, 1 << 20) == size_class(2_000_000, (1 << 20) + 5)
    assert size_class(1920 * 1080, 1 << 20) != size_class(1920 * 1080, 1 << 21)
    assert size_class(0, 0) == "l1_e1"


def test_tune_once_then_cached(tmp_path):
    path = str(tmp_path / "tune.json")
    ctx = FakeCtx()
    at = Autotuner(ctx, cache_path=path, sample_eyes=1000)
    e = at.tune(*_eyes(5000), None, 1.0, n_lights=70000)
    assert ctx.calls == [1000]  # tuned on the bounded sample
    assert Autotuner.launch_fields(e) == {"rangemin_variant": 2, "blocks_per_sm": 5, "node_width": 4,
                                          "ring_entries": 256, "threads_per_block": 128}
    assert e["sample_ms"] == 1.25  # the fastest candidate of the table
    assert len(at.last_table) == 3
    again = at.tune(*_eyes(6000), None, 1.0, n_lights=66000)  # same class
    assert again == e and ctx.calls == [1000]
    at.tune(*_eyes(500), None, 1.0, n_lights=70000)  # new class, smaller than the sample
    assert ctx.calls == [1000, 500]
    with open(path) as f:
        table = json.load(f)
    assert set(table) == {size_class(5000, 70000), size_class(500, 70000)}
    # a fresh tuner reads the cache and does not tune again
    ctx2 = FakeCtx()
    at2 = Autotuner(ctx2, cache_path=path)
    assert at2.tune(*_eyes(4100), None, 1.0, n_lights=65600) == e and ctx2.calls == []


def test_launch_fields_of_missing_entry():
    assert Autotuner.launch_fields(None) is None
    assert Autotuner(FakeCtx()).get(10, 10) is None
