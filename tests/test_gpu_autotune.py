"""The traversal's tuning changes its speed only: every tuning the autotuner can pick gives
the same accepted set, every tuning of one node width the same per-eye visit counts (those
of the oracle's traversal read with that width), and hrr_autotune returns one of the
timed candidates."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import default_width, dev, oracle_hier, sorted_pairs, upload_scene

pytestmark = pytest.mark.gpu


def test_autotune_returns_a_candidate_and_all_tunings_agree(tmp_path):
    import torch

    import paper_1907_12343_gb300 as hrr
    from paper_1907_12343_gb300.autotune import Autotuner
    ctx = hrr.Context(0)
    s = synth.scene_frame(width=257, height=131, n_lights=50021, tile_w=64, tile_h=64,
                          target=64.0, seed=7)
    g = upload_scene(s)
    ctx.set_shift_tile(s["tile"])
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    tau = float(s["tau"])
    at = Autotuner(ctx, cache_path=str(tmp_path / "t.json"), sample_eyes=8192)
    best = at.tune(g["ex"], g["ey"], g["ez"], g["px"], g["py"], tree, tau, n_lights=50021)
    assert best["rangemin_variant"] in (0, 2) and best["node_width"] in (2, 4)
    assert best["threads_per_block"] in (128, 256) and best["sample_ms"] > 0
    table = at.last_table
    assert len(table) >= 32 and all(ms > 0 for _, ms in table)
    assert Autotuner.launch_fields(best) in [t for t, _ in table]
    assert best["sample_ms"] == min(ms for _, ms in table)
    n = g["ex"].numel()
    t_or = oracle.Tree(s.light_pos, s.intensity)
    want_vis = {w: oracle_hier(t_or, s.eye_pos, s.px, s.py, s.tile, s.tau, width=w)["visits"].astype(np.uint32)
                for w in (2, 4)}
    ref_pairs = None
    tunings = [None, Autotuner.launch_fields(best), {"rangemin_variant": 2, "blocks_per_sm": 2},
               {"rangemin_variant": 0, "blocks_per_sm": 1, "node_width": 2},
               {"rangemin_variant": 2, "blocks_per_sm": 3, "node_width": 4, "ring_entries": 512}]
    tunings += [t for t, _ in table[::5]]
    for t in tunings:
        pairs = torch.empty((256 * n, 2), dtype=torch.int32, device=dev())
        vis = torch.zeros(n, dtype=torch.int32, device=dev())
        st, cnt = ctx.cull(g["ex"], g["ey"], g["ez"], g["px"], g["py"], tree, tau, pairs, eye_visits=vis,
                           tuning=t)
        assert st == hrr.HRR_OK
        got = sorted_pairs(pairs[:cnt].cpu().numpy().view(np.uint32))
        if ref_pairs is None:
            ref_pairs = got
        assert np.array_equal(got, ref_pairs)
        w = (t or {}).get("node_width") or default_width()
        assert np.array_equal(vis.cpu().numpy().view(np.uint32), want_vis[w]), t
    tree.free()
    ctx.close()
