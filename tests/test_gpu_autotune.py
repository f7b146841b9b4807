"""The traversal's launch shape changes its speed only: every tuning the autotuner can pick
gives the same accepted set and the same per-eye visit counts, and hrr_autotune returns
one of the candidates."""
import numpy as np
import pytest

import synth
from gpu_util import dev, sorted_pairs, upload_scene

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
    assert best["rangemin_variant"] in (0, 2)
    assert best["blocks_per_sm"] in (4, 5, 6)
    assert best["sample_ms"] > 0
    n = g["ex"].numel()
    ref = None
    for t in [None, Autotuner.launch_fields(best), {"rangemin_variant": 2, "blocks_per_sm": 2},
              {"rangemin_variant": 0, "blocks_per_sm": 1}, {"rangemin_variant": 2, "blocks_per_sm": 3}]:
        pairs = torch.empty((256 * n, 2), dtype=torch.int32, device=dev())
        vis = torch.zeros(n, dtype=torch.int32, device=dev())
        st, cnt = ctx.cull(g["ex"], g["ey"], g["ez"], g["px"], g["py"], tree, tau, pairs, eye_visits=vis,
                           tuning=t)
        assert st == hrr.HRR_OK
        got = (sorted_pairs(pairs[:cnt].cpu().numpy().view(np.uint32)), vis.cpu().numpy())
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    tree.free()
    ctx.close()
