"""Traversals whose pending-node stack outgrows the shared-memory ring, so that entries
move to the spill area in global memory and back: nothing culled (every pair accepted,
every internal node visited), and a workload with thousands of accepted lights per eye,
against the oracle; also inside a batch."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, oracle_hier, run_cull, sorted_pairs, upload_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("width", [2, 4])
def test_nothing_culled_visits_every_node(ctx, width):
    # full traversal of a 2^18-light tree: the pending frontier exceeds the ring, so the
    # stack spills to global memory and comes back (its bound sizes the spill area)
    s = dict(synth.scene_frame(width=8, height=6, n_lights=1 << 18, tile_w=8, tile_h=8, seed=21))
    s["tau"] = np.float32(1e30)
    g = upload_scene(s)
    ctx.set_shift_tile(s["tile"])
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    n_e, n_l = len(s["eye_pos"]), len(s["light_pos"])
    st, cnt, pairs, vis = run_cull(ctx, g, tree, float(s["tau"]), cap=n_e * n_l, visits=True,
                                   tuning={"node_width": width})
    tree.free()
    assert st == 0 and cnt == n_e * n_l
    if width == 2:
        assert np.all(vis == n_l - 1)
    else:  # every even-depth internal node
        t = oracle.Tree(s["light_pos"], s["intensity"])
        one = oracle_hier(t, s["eye_pos"][:1], s["px"][:1], s["py"][:1], s["tile"], s["tau"], width=4)
        assert np.all(vis == int(one["visits"][0])) and n_l // 4 < int(one["visits"][0]) < n_l // 2
    p = sorted_pairs(pairs)
    assert np.array_equal(p[:, 0], np.repeat(np.arange(n_e, dtype=np.uint32), n_l))
    assert np.array_equal(p[:, 1], np.tile(np.arange(n_l, dtype=np.uint32), n_e))


@pytest.mark.parametrize("width", [2, 4])
def test_thousands_accepted_per_eye_equal_oracle(ctx, width):
    s = synth.scene_frame(width=9, height=5, n_lights=1 << 18, tile_w=8, tile_h=8, target=6000.0, seed=22)
    g = upload_scene(s)
    ctx.set_shift_tile(s.tile)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    st, cnt, pairs, vis = run_cull(ctx, g, tree, float(s.tau), cap=len(s.eye_pos) * 20000, visits=True,
                                   tuning={"node_width": width})
    tree.free()
    assert st == 0
    t = oracle.Tree(s.light_pos, s.intensity)
    hier = oracle_hier(t, s.eye_pos, s.px, s.py, s.tile, s.tau, width=width)
    assert cnt == len(hier["pairs"]) and cnt > 1000 * len(s.eye_pos)
    assert np.array_equal(sorted_pairs(pairs), sorted_pairs(hier["pairs"]))
    assert np.array_equal(vis, hier["visits"].astype(np.uint32))


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_with_a_full_traversal_frame(ctx, use_graph):
    import torch

    import paper_1907_12343_gb300 as hrr
    full = dict(synth.scene_frame(width=4, height=4, n_lights=1 << 17, tile_w=8, tile_h=8, seed=23))
    full["tau"] = np.float32(1e30)
    normal = dict(synth.scene_frame(width=33, height=17, n_lights=20000, tile_w=16, tile_h=16, seed=24))
    frames, want = [], []
    for s in (full, normal, full):
        g = upload_scene(s)
        tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
        n = g["ex"].numel()
        ctx.set_shift_tile(s["tile"])
        st, cnt, pairs, vis = run_cull(ctx, g, tree, float(s["tau"]), cap=n * len(s["light_pos"]), visits=True)
        assert st == 0
        want.append((cnt, sorted_pairs(pairs), vis))
        frames.append({"x": g["ex"], "y": g["ey"], "z": g["ez"], "px": g["px"], "py": g["py"], "tree": tree,
                       "tau": float(s["tau"]),
                       "tile": torch.from_numpy(np.ascontiguousarray(s["tile"]).view(np.int32)).to(dev()),
                       "pairs": torch.empty((cnt + 64, 2), dtype=torch.int32, device=dev()),
                       "eye_visits": torch.zeros(n, dtype=torch.int32, device=dev())})
    b = hrr.Batch(ctx, frames, use_graph=use_graph)
    for _ in range(2):
        b.launch()
        st, counts, _ = b.results()
        assert st == hrr.HRR_OK
        for fr, (cnt, pairs, vis), got in zip(frames, want, counts):
            assert got == cnt
            p = fr["pairs"][:cnt].cpu().numpy().view(np.uint32)
            assert np.array_equal(sorted_pairs(p), pairs)
            assert np.array_equal(fr["eye_visits"].cpu().numpy().view(np.uint32), vis)
    b.destroy()
    for fr in frames:
        fr["tree"].free()
