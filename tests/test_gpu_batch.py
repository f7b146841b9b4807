"""Batched culling through the C ABI: every frame of a batch gets exactly what a plain
hrr_cull of that frame gets (connection set and per-eye visits), whether the batch runs
as a recorded CUDA graph or not, on replays, and alongside frames of very different sizes."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, run_cull, sorted_pairs, upload_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    yield c
    c.close()


def _scenes():
    s1 = dict(synth.scene_frame(width=257, height=131, n_lights=50021, tile_w=64, tile_h=64,
                                target=64.0, seed=7))
    s2 = dict(synth.scene_uniform())
    s3 = dict(synth.scene_frame(width=61, height=37, n_lights=5003, tile_w=16, tile_h=16,
                                target=48.0, seed=5))
    one = dict(synth.scene_uniform(n_lights=64, grid_w=16, grid_h=8, tile_w=8, tile_h=8,
                                   target=4.0, seed=9))
    one["light_pos"], one["intensity"] = one["light_pos"][:1], one["intensity"][:1]
    one["tau"] = np.float32(one["tau"] * 20)
    empty = dict(synth.scene_uniform(n_lights=300, grid_w=8, grid_h=4, tile_w=8, tile_h=8, seed=10))
    empty["eye_pos"], empty["px"], empty["py"] = empty["eye_pos"][:0], empty["px"][:0], empty["py"][:0]
    return [s1, s2, s3, one, empty]


def _frame(ctx, s, cap, shift_offset=0):
    import torch
    g = upload_scene(s)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    n = g["ex"].numel()
    tile = torch.from_numpy(np.ascontiguousarray(s["tile"]).view(np.int32)).to(dev())
    return {"x": g["ex"], "y": g["ey"], "z": g["ez"], "px": g["px"], "py": g["py"], "tree": tree,
            "tau": float(s["tau"]), "tile": tile, "shift_offset": shift_offset,
            "pairs": torch.empty((cap, 2), dtype=torch.int32, device=dev()),
            "eye_visits": torch.zeros(max(n, 1), dtype=torch.int32, device=dev()), "_g": g, "_s": s}


def _plain(ctx, fr):
    ctx.set_shift_tile(fr["_s"]["tile"])
    n = fr["x"].numel()
    st, cnt, pairs, vis = run_cull(ctx, fr["_g"], fr["tree"], fr["tau"], visits=n > 0,
                                   shift_offset=fr["shift_offset"])
    return st, pairs, vis


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_plain_per_frame(ctx, use_graph):
    import paper_1907_12343_gb300 as hrr
    frames = [_frame(ctx, s, cap=max(1024, 256 * len(s["eye_pos"])), shift_offset=o)
              for s, o in zip(_scenes(), [0, 0x9E3779B9, 0, 7, 0])]
    b = hrr.Batch(ctx, frames, use_graph=use_graph)
    for rep in range(2):  # a replay must reset the counters
        b.launch()
        st, counts, visits = b.results()
        assert st == hrr.HRR_OK
        for fr, cnt, v in zip(frames, counts, visits):
            n = fr["x"].numel()
            got = fr["pairs"][:cnt].cpu().numpy().view(np.uint32)
            if rep == 1:
                continue
            pst, ref, ref_vis = _plain(ctx, fr)
            assert pst == hrr.HRR_OK
            assert np.array_equal(sorted_pairs(got), sorted_pairs(ref))
            if n:
                ev = fr["eye_visits"][:n].cpu().numpy().view(np.uint32)
                assert np.array_equal(ev, ref_vis)
                assert v == int(ref_vis.sum())
            else:
                assert cnt == 0 and v == 0
    # the first (uniform) scene also against the flat oracle
    s = frames[1]["_s"]
    t = oracle.Tree(s["light_pos"], s["intensity"])
    tile = (s["tile"].astype(np.uint64) + 0x9E3779B9).astype(np.uint32)
    flat = oracle.cull_flat(t, s["eye_pos"], s["px"], s["py"], tile, s["tau"])
    got = frames[1]["pairs"][:counts[1]].cpu().numpy().view(np.uint32)
    assert np.array_equal(sorted_pairs(got), sorted_pairs(flat["pairs"]))
    b.destroy()
    for fr in frames:
        fr["tree"].free()


def test_batch_overflow_is_per_frame(ctx):
    import paper_1907_12343_gb300 as hrr
    scenes = _scenes()[:3]
    frames = [_frame(ctx, s, cap=max(1024, 256 * len(s["eye_pos"]))) for s in scenes]
    frames[1]["pairs"] = frames[1]["pairs"][:100]
    b = hrr.Batch(ctx, frames, use_graph=True)
    b.launch()
    st, counts, _ = b.results()
    assert st == hrr.HRR_ERR_OVERFLOW
    assert counts[1] > 100
    st0, ref0, _ = _plain(ctx, frames[0])
    assert np.array_equal(sorted_pairs(frames[0]["pairs"][:counts[0]].cpu().numpy().view(np.uint32)),
                          sorted_pairs(ref0))
    b.destroy()
    for fr in frames:
        fr["tree"].free()


def test_batch_validation(ctx):
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)  # no context tile
    s = _scenes()[1]
    fr = _frame(c, s, cap=4096)
    fr_no_tile = dict(fr)
    fr_no_tile["tile"] = None
    with pytest.raises(hrr.HRRError) as e:
        hrr.Batch(c, [fr_no_tile])
    assert e.value.status == hrr.HRR_ERR_NO_TILE
    bad = dict(fr)
    bad["tau"] = float("nan")
    with pytest.raises(hrr.HRRError) as e:
        hrr.Batch(c, [fr, bad])
    assert e.value.status == hrr.HRR_ERR_INVALID_ARG
    fr["tree"].free()
    c.close()


def test_more_frames_than_one_launch_holds(ctx):
    # 300 frames (three launches of at most 128 frames) over two shared hierarchies, each
    # frame with its own sample offset: every frame equals its plain cull
    import torch

    import paper_1907_12343_gb300 as hrr
    scenes = [dict(synth.scene_uniform(n_lights=700, grid_w=8, grid_h=8, tile_w=8, tile_h=8, seed=31)),
              dict(synth.scene_frame(width=12, height=7, n_lights=3001, tile_w=16, tile_h=16, seed=32))]
    up = []
    for s in scenes:
        g = upload_scene(s)
        up.append((s, g, ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"]),
                   torch.from_numpy(np.ascontiguousarray(s["tile"]).view(np.int32)).to(dev())))
    frames, want = [], []
    for k in range(300):
        s, g, tree, tile = up[k % 2]
        off = (k * 0x9E3779B9) & 0xFFFFFFFF
        ctx.set_shift_tile(s["tile"])
        st, cnt, pairs, _ = run_cull(ctx, g, tree, float(s["tau"]), shift_offset=off)
        assert st == 0
        want.append(sorted_pairs(pairs))
        frames.append({"x": g["ex"], "y": g["ey"], "z": g["ez"], "px": g["px"], "py": g["py"], "tree": tree,
                       "tau": float(s["tau"]), "tile": tile, "shift_offset": off,
                       "pairs": torch.empty((cnt + 8, 2), dtype=torch.int32, device=dev())})
    launches0 = ctx.launch_count()
    b = hrr.Batch(ctx, frames, use_graph=True)
    b.launch()
    st, counts, _ = b.results()
    assert st == hrr.HRR_OK
    assert ctx.launch_count() - launches0 == 3
    for fr, w, c in zip(frames, want, counts):
        assert c == len(w)
        assert np.array_equal(sorted_pairs(fr["pairs"][:c].cpu().numpy().view(np.uint32)), w)
    b.destroy()
    for _, _, tree, _ in up:
        tree.free()


def test_new_context_tile_leaves_batch_and_job_on_their_tile(ctx):
    # A batch (recorded graph) and a served job that read the context's tile keep reading
    # the tile they were created with after hrr_set_shift_tile replaces it: the old tile
    # stays alive (reference-counted) until the batch is destroyed and the job released.
    import torch
    import paper_1907_12343_gb300 as hrr
    s = _scenes()[2]
    fr = _frame(ctx, s, cap=256 * len(s["eye_pos"]))
    fr.pop("tile")  # the frame reads the context tile
    ctx.set_shift_tile(s["tile"])
    pst, ref, ref_vis = _plain(ctx, fr)
    assert pst == hrr.HRR_OK
    b = hrr.Batch(ctx, [fr], use_graph=True)
    srv = hrr.Server(ctx, 1 << 30, max_jobs=4)
    other = (np.asarray(s["tile"], np.uint32) ^ np.uint32(0x5A5A5A5A)).astype(np.uint32)
    t = srv.submit(fr["x"], fr["y"], fr["z"], fr["px"], fr["py"], fr["tree"], fr["tau"], len(ref) + 1024)
    ctx.set_shift_tile(other)   # replaces (and would have freed) the tile both still use
    torch.cuda.synchronize()
    for _ in range(2):
        b.launch()
        st, counts, _ = b.results()
        assert st == hrr.HRR_OK
        got = fr["pairs"][:counts[0]].cpu().numpy().view(np.uint32)
        assert np.array_equal(sorted_pairs(got), sorted_pairs(ref))
    r = srv.wait(t, 60.0)
    assert r["status"] == hrr.HRR_OK and r["count"] == len(ref)
    host = srv.pairs(t, r)
    assert np.array_equal(sorted_pairs(host), sorted_pairs(ref))
    srv.release(t)
    srv.destroy()
    b.destroy()
    # the context now culls with the new tile: a different set
    st2, cnt2, pairs2, _ = run_cull(ctx, fr["_g"], fr["tree"], fr["tau"])
    assert st2 == hrr.HRR_OK
    assert not np.array_equal(sorted_pairs(pairs2), sorted_pairs(ref))
    fr["tree"].free()


@pytest.mark.parametrize("use_graph", [True, False])
def test_mixed_batch_own_and_shared_launches(ctx, use_graph):
    # frames with at least 2^16 eyes run as launches of their own (the single-frame kernel,
    # alternating streams), the small ones between them share batched launches; every frame
    # gets exactly its plain result, on replays too
    import paper_1907_12343_gb300 as hrr
    big_a = dict(synth.scene_frame(width=256, height=256, n_lights=20011, tile_w=64, tile_h=64,
                                   target=32.0, seed=61))
    big_b = dict(synth.scene_frame(width=320, height=240, n_lights=7001, tile_w=16, tile_h=16,
                                   target=16.0, seed=62))
    smalls = _scenes()[:3]
    order = [big_a, smalls[0], smalls[1], big_b, smalls[2], big_a]
    frames = [_frame(ctx, s, cap=max(1024, 160 * len(s["eye_pos"]))) for s in order]
    b = hrr.Batch(ctx, frames, use_graph=use_graph)
    for rep in range(2):
        b.launch()
        st, counts, visits = b.results()
        assert st == hrr.HRR_OK
        for fr, cnt, v in zip(frames, counts, visits):
            got = fr["pairs"][:cnt].cpu().numpy().view(np.uint32)
            if rep == 0:
                pst, ref, ref_vis = _plain(ctx, fr)
                fr["_ref"] = (sorted_pairs(ref), int(ref_vis.sum()))
            assert np.array_equal(sorted_pairs(got), fr["_ref"][0])
            assert v == fr["_ref"][1]
    b.destroy()
    for fr in frames:
        fr["tree"].free()
