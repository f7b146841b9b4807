"""Per-size-class autotuning of the traversal's form and launch shape, cached in JSON.

The traversal gives identical results for every tuning (range-minimum variant, node
width, top levels evaluated from shared memory, shared-memory stack ring, threads per
block, resident blocks per SM); only its speed depends on the workload.
``Autotuner`` keys workloads by size class (bit lengths of N_l and N_e), tunes a class
once on a sample of its eyes with ``hrr_autotune`` and stores the answer, so later
frames, batches and servers of that class reuse it.
"""
from __future__ import annotations

import json
import os


def size_class(n_eyes: int, n_lights: int) -> str:
    """Workloads whose light and eye counts have the same bit lengths share a class."""
    return f"l{max(int(n_lights), 1).bit_length()}_e{max(int(n_eyes), 1).bit_length()}"


class Autotuner:
    def __init__(self, ctx, cache_path: str | None = None, sample_eyes: int = 1 << 19):
        self.ctx = ctx
        self.path = cache_path
        self.sample = sample_eyes
        self.table: dict[str, dict] = {}
        self.last_table: list = []  # every candidate's (tuning, ms) of the last tuning run
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.table = json.load(f)

    def get(self, n_eyes: int, n_lights: int):
        return self.table.get(size_class(n_eyes, n_lights))

    def put(self, n_eyes: int, n_lights: int, tuning: dict, ms: float | None = None):
        entry = dict(tuning)
        if ms is not None:
            entry["sample_ms"] = ms
        self.table[size_class(n_eyes, n_lights)] = entry
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        return entry

    def tune(self, x, y, z, px, py, tree, tau, n_lights: int):
        """Tune (or reuse) the class of a frame; the sample is its first eyes."""
        n_eyes = int(x.numel())
        hit = self.get(n_eyes, n_lights)
        if hit is not None:
            return hit
        import torch
        k = min(n_eyes, self.sample)
        pairs = torch.empty((max(k * 256, 1024), 2), dtype=torch.int32, device=x.device)
        table = self.ctx.autotune_all(x[:k], y[:k], z[:k], px[:k], py[:k], tree, tau, pairs)
        tuning, ms = min(table, key=lambda tm: tm[1])
        entry = self.put(n_eyes, n_lights, tuning, ms)
        self.last_table = table
        return entry

    @staticmethod
    def launch_fields(entry: dict | None) -> dict | None:
        if entry is None:
            return None
        from . import TUNING_FIELDS
        return {k: entry[k] for k in TUNING_FIELDS if k in entry}
