"""GPU parity of hierarchical Russian-roulette culling (Sec. 1) through the C ABI.

The accepted (eye, light) set must equal the oracle's flat brute force exactly (the float32
acceptance expression is evaluated in the same order on both sides); per-eye node-visit
counts must equal the oracle's hierarchical traversal over the same radix tree.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import oracle_hier, run_cull, sorted_pairs, upload_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    yield c
    c.close()


def _gpu(ctx, s, **kw):
    g = upload_scene(s)
    ctx.set_shift_tile(s["tile"])
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    res = run_cull(ctx, g, tree, float(s["tau"]), **kw)
    tree.free()
    return res


# every compiled form: node width, stack ring, threads per block, and for binary records the
# top levels evaluated from shared memory (1: walked from the root)
FORMS = [{"node_width": w, "ring_entries": r, "threads_per_block": th, "top_levels": top}
         for w, rings, tops in ((2, (128, 256), (1, 6)), (4, (256, 512), (1,)))
         for r in rings for th in (128, 256) for top in tops]
FORM_ID = "w{node_width}r{ring_entries}t{threads_per_block}top{top_levels}".format
# the node width and top levels alone (the other fields at their defaults)
SHAPES = [{"node_width": 2, "top_levels": 1}, {"node_width": 2, "top_levels": 6}, {"node_width": 4}]
SHAPE_ID = lambda f: "w{}top{}".format(f["node_width"], f.get("top_levels", 1))


@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("form", FORMS, ids=lambda f: FORM_ID(**f))
def test_uniform_tiny_scene_equals_flat(ctx, variant, form):
    # 1024 eyes x 4096 lights, 32x32 tile, tau for ~32 accepted per eye, in every compiled
    # form of the traversal (node width, stack ring, threads per block)
    s = synth.scene_uniform()
    st, cnt, pairs, vis = _gpu(ctx, s, visits=True, tuning=dict(form, rangemin_variant=variant))
    assert st == 0
    t = oracle.Tree(s.light_pos, s.intensity)
    flat = oracle.cull_flat(t, s.eye_pos, s.px, s.py, s.tile, s.tau)
    assert np.array_equal(sorted_pairs(pairs), sorted_pairs(flat["pairs"]))
    hier = oracle_hier(t, s.eye_pos, s.px, s.py, s.tile, s.tau, width=form["node_width"])
    assert np.array_equal(vis, hier["visits"].astype(np.uint32))
    v_total, acc = ctx.last_cull_stats()
    assert v_total == hier["total_visits"] and acc == cnt == len(flat["pairs"])


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_ID)
def test_ragged_frame_equals_oracle(ctx, shape):
    # eye count not a multiple of the warp or block size, light count not a power of two
    s = synth.scene_frame(width=257, height=131, n_lights=50021, tile_w=64, tile_h=64,
                          target=64.0, seed=7)
    width = shape["node_width"]
    st, cnt, pairs, vis = _gpu(ctx, s, visits=True, tuning=shape)
    assert st == 0
    t = oracle.Tree(s.light_pos, s.intensity)
    hier = oracle_hier(t, s.eye_pos, s.px, s.py, s.tile, s.tau, width=width)
    assert np.array_equal(sorted_pairs(pairs), sorted_pairs(hier["pairs"]))
    assert np.array_equal(vis, hier["visits"].astype(np.uint32))
    # flat brute force on a sample of eyes (hier == flat is pinned on the CPU)
    ids = np.arange(0, len(s.eye_pos), 97, dtype=np.uint32)
    flat = oracle.cull_flat(t, s.eye_pos[ids], s.px[ids], s.py[ids], s.tile, s.tau, eye_ids=ids)
    got = pairs[np.isin(pairs[:, 0], ids)]
    assert np.array_equal(sorted_pairs(got), sorted_pairs(flat["pairs"]))


def test_full_size_frame_sampled(ctx):
    # 1920x1080 eyes x 2^20 lights in the launch configuration used for timing; sampled
    # eyes are compared with the flat brute force and the hierarchical oracle
    s = synth.scene_frame()
    cap = 200_000_000
    st, cnt, pairs, vis = _gpu(ctx, s, cap=cap, visits=True)
    assert st == 0 and cnt <= cap
    n_e = len(s.eye_pos)
    assert 20 * n_e < cnt < 200 * n_e  # about 64 accepted per eye
    ids = np.unique(np.concatenate([np.arange(0, n_e, n_e // 301), [n_e - 1]])).astype(np.uint32)
    t = oracle.Tree(s.light_pos, s.intensity)
    hier = oracle_hier(t, s.eye_pos[ids], s.px[ids], s.py[ids], s.tile, s.tau, eye_ids=ids)
    got = pairs[np.isin(pairs[:, 0], ids)]
    assert np.array_equal(sorted_pairs(got), sorted_pairs(hier["pairs"]))
    assert np.array_equal(vis[ids], hier["visits"].astype(np.uint32))
    few = ids[::10]
    flat = oracle.cull_flat(t, s.eye_pos[few], s.px[few], s.py[few], s.tile, s.tau, eye_ids=few)
    assert np.array_equal(sorted_pairs(pairs[np.isin(pairs[:, 0], few)]), sorted_pairs(flat["pairs"]))
    # every eye index appears within range; per-eye counts add up
    assert pairs[:, 0].max() < n_e
    assert np.bincount(pairs[:, 0], minlength=n_e).sum() == cnt


def test_largest_batch_frame_sampled(ctx):
    # the largest frame of the batched workload: 1920 x 1080 eyes x 2^22 lights at 128
    # accepted per eye, over the cost-driven hierarchy; sampled eyes equal the
    # hierarchical oracle (pairs and visits), and the count stays within the per-eye cap
    s = synth.scene_frame(width=1920, height=1080, n_lights=1 << 22, target=128.0, seed=41, tau_lights=1 << 18)
    g = upload_scene(s)
    ctx.set_shift_tile(s.tile)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology="cost")
    import torch
    n_e = len(s.eye_pos)
    cap = 300 * n_e
    pairs = torch.empty((cap, 2), dtype=torch.int32, device=g["ex"].device)
    vis = torch.zeros(n_e, dtype=torch.int32, device=g["ex"].device)
    st, cnt = ctx.cull(g["ex"], g["ey"], g["ez"], g["px"], g["py"], tree, float(s.tau), pairs, eye_visits=vis)
    tree.free()
    assert st == 0 and 60 * n_e < cnt < cap
    ids = np.unique(np.concatenate([np.arange(0, n_e, n_e // 151), [n_e - 1]])).astype(np.uint32)
    sel = pairs[:cnt][torch.isin(pairs[:cnt, 0], torch.from_numpy(ids.astype(np.int32)).to(pairs.device))]
    got = sel.cpu().numpy().view(np.uint32)
    del pairs, sel
    t = oracle.Tree(s.light_pos, s.intensity, topology="cost")
    hier = oracle_hier(t, s.eye_pos[ids], s.px[ids], s.py[ids], s.tile, s.tau, eye_ids=ids)
    assert np.array_equal(sorted_pairs(got), sorted_pairs(hier["pairs"]))
    assert np.array_equal(vis.cpu().numpy().view(np.uint32)[ids], hier["visits"].astype(np.uint32))


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_ID)
@pytest.mark.parametrize("n_lights", [1, 2, 3, 4, 5, 33, 63, 64, 65])
def test_tiny_light_sets(ctx, n_lights, shape):
    # trees whose top levels hold leaves and empty slots (up to 63 lights: all of the tree)
    s = dict(synth.scene_uniform(n_lights=65, grid_w=16, grid_h=8, tile_w=8, tile_h=8,
                                 target=4.0, seed=9))
    s["light_pos"] = s["light_pos"][:n_lights]
    s["intensity"] = s["intensity"][:n_lights]
    s["tau"] = np.float32(s["tau"] * 20)
    width = shape["node_width"]
    st, cnt, pairs, vis = _gpu(ctx, s, visits=True, tuning=shape)
    assert st == 0
    t = oracle.Tree(s["light_pos"], s["intensity"])
    flat = oracle.cull_flat(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"])
    hier = oracle_hier(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"], width=width)
    assert np.array_equal(sorted_pairs(pairs), sorted_pairs(flat["pairs"]))
    assert np.array_equal(vis, hier["visits"].astype(np.uint32))


@pytest.mark.parametrize("topology", ["radix", "cost"])
@pytest.mark.parametrize("top", [1, 6])
def test_leaves_near_the_root(ctx, top, topology):
    # lights at x = 2^-1 .. 2^-21 beside a dense cluster at the origin: the radix tree cuts
    # them off one by one (leaves at depths 1, 3, 4 and 5), the cost-driven tree at depths
    # 4 and 5, so the top levels mix leaves, internal nodes and empty slots; pairs equal the
    # flat oracle and visits the hierarchical one
    rng = np.random.default_rng(5)
    x = (2.0 ** -np.arange(1, 22, dtype=np.float64)).astype(np.float32)
    line = np.stack([x, np.full_like(x, 0.5), np.full_like(x, 0.5)], axis=1)
    pos = np.concatenate([line, (rng.random((3000, 3)) * 1e-3).astype(np.float32)]).astype(np.float32)
    inten = np.ones(len(pos), np.float32)
    s = dict(synth.scene_uniform(n_lights=16, grid_w=32, grid_h=16, tile_w=16, tile_h=16, seed=13))
    s["light_pos"], s["intensity"], s["tau"] = pos, inten, np.float32(1e-3)
    g = upload_scene(s)
    ctx.set_shift_tile(s["tile"])
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology=topology)
    st, cnt, pairs, vis = run_cull(ctx, g, tree, float(s["tau"]), visits=True,
                                   tuning={"node_width": 2, "top_levels": top})
    tree.free()
    assert st == 0 and cnt > 0
    t = oracle.Tree(pos, inten, topology=topology)
    flat = oracle.cull_flat(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"])
    hier = oracle_hier(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"], width=2)
    assert np.array_equal(sorted_pairs(pairs), sorted_pairs(flat["pairs"]))
    assert np.array_equal(vis, hier["visits"].astype(np.uint32))


def test_zero_eyes_and_extreme_tau(ctx):
    s = dict(synth.scene_uniform(n_lights=300, grid_w=8, grid_h=4, tile_w=8, tile_h=8, seed=10))
    st, cnt, pairs, _ = _gpu(ctx, s, n_eyes=0)
    assert st == 0 and cnt == 0
    s["tau"] = np.float32(0.0)
    st, cnt, _, _ = _gpu(ctx, s)
    assert st == 0 and cnt == 0
    s["tau"] = np.float32(1e30)
    st, cnt, pairs, _ = _gpu(ctx, s, cap=32 * 300)
    assert st == 0 and cnt == 32 * 300
    assert set(map(tuple, pairs.tolist())) == {(j, i) for j in range(32) for i in range(300)}


def test_overflow_reports_need_and_retry_succeeds(ctx):
    import paper_1907_12343_gb300 as hrr
    s = synth.scene_uniform()
    st, need, _, _ = _gpu(ctx, s, cap=1000)
    assert st == hrr.HRR_ERR_OVERFLOW and need > 1000
    st, cnt, pairs, _ = _gpu(ctx, s, cap=need)
    assert st == 0 and cnt == need
    t = oracle.Tree(s.light_pos, s.intensity)
    flat = oracle.cull_flat(t, s.eye_pos, s.px, s.py, s.tile, s.tau)
    assert np.array_equal(sorted_pairs(pairs), sorted_pairs(flat["pairs"]))


def test_shift_offset_is_absorbed_into_the_shift(ctx):
    # Sec. 3: a sample offset psi(n) adds to every eye's shift; the culling result equals
    # the plain method run with the tile rotated by psi(n)
    s = dict(synth.scene_uniform(n_lights=2000, grid_w=16, grid_h=16, tile_w=16, tile_h=16, seed=11))
    psi = 0x9E3779B9  # golden-ratio lattice step 1/phi in 32-bit fixed point
    st, cnt, pairs, _ = _gpu(ctx, s, shift_offset=psi)
    assert st == 0
    t = oracle.Tree(s["light_pos"], s["intensity"])
    tile = (s["tile"].astype(np.uint64) + psi).astype(np.uint32)
    flat = oracle.cull_flat(t, s["eye_pos"], s["px"], s["py"], tile, s["tau"])
    assert np.array_equal(sorted_pairs(pairs), sorted_pairs(flat["pairs"]))


def test_missing_tile_and_bad_tau(ctx):
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    s = synth.scene_uniform(n_lights=100, grid_w=4, grid_h=4, tile_w=4, tile_h=4, seed=12)
    g = upload_scene(s)
    tree = c.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    with pytest.raises(hrr.HRRError) as e:
        run_cull(c, g, tree, float(s.tau))
    assert e.value.status == hrr.HRR_ERR_NO_TILE
    c.set_shift_tile(s.tile)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(hrr.HRRError) as e:
            run_cull(c, g, tree, bad)
        assert e.value.status == hrr.HRR_ERR_INVALID_ARG
    tree.free()
    c.close()
