"""The cost-driven hierarchy (HRR_TOPOLOGY_COST) built on the GPU equals the oracle's
node by node (splits, ranges, boxes, maximum intensities, permutation, height), and
culling over it is exact (connection sets and per-eye visits)."""
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


def _records_equal(tree, t):
    nodes, perm = tree.download()
    assert np.array_equal(perm, t.perm)
    assert tree.height == t.height
    n = t.n
    if n == 1:
        return
    first = np.minimum(np.arange(n - 1), nodes["other_end"])
    last = np.maximum(np.arange(n - 1), nodes["other_end"])
    assert np.array_equal(first, t.first) and np.array_equal(last, t.last)
    assert np.array_equal(nodes["split"], t.split)
    s = nodes["split"].astype(np.int64)
    for c, cid, leaf in ((0, s, first == s), (1, s + 1, last == s + 1)):
        lo, hi, im = nodes[f"c{c}_lo"], nodes[f"c{c}_hi"], nodes[f"c{c}_imax"]
        li, ii = cid[leaf], cid[~leaf]
        assert np.array_equal(lo[leaf], t.pos[li]) and np.array_equal(hi[leaf], t.pos[li])
        assert np.array_equal(im[leaf], t.inten[li])
        assert np.array_equal(lo[~leaf], t.lo[ii]) and np.array_equal(hi[~leaf], t.hi[ii])
        assert np.array_equal(im[~leaf], t.imax[ii])


def _lights(pos, inten):
    g = upload_scene({"light_pos": pos, "intensity": inten, "eye_pos": pos[:1], "px": np.zeros(1, np.uint16),
                      "py": np.zeros(1, np.uint16)})
    return g["lx"], g["ly"], g["lz"], g["li"]


@pytest.mark.parametrize("case", ["n2", "n3", "n33", "n257", "n1000", "n1025", "n5000", "n100003", "n600001",
                                  "n4194304", "duplicates", "dark", "chain", "depth1", "depth3"])
def test_cost_tree_equals_oracle(ctx, case):
    # 33 / 257 / 1025 lights: the first range of each split kernel (warp run of 8, one tile,
    # two tiles); 600001 lights: 587 tiles at the root, scanned in three block passes;
    # depth1 / depth3: radix splits below a shallow cost depth; 2^22 lights: the largest
    # light set of the batched workload
    n = {"n2": 2, "n3": 3, "n33": 33, "n257": 257, "n1000": 1000, "n1025": 1025, "n5000": 5000,
         "n100003": 100003, "n600001": 600001, "n4194304": 1 << 22}.get(case, 20000)
    depth = {"depth1": 1, "depth3": 3}.get(case, 0)
    if n > 1 << 20:  # the frame recipe's lights and intensities, without its tau calibration
        pos = synth.gaussian_mixture_lights(n, 64, 101)
        inten = np.exp(1.5 * synth.normal(101, 21, n)).astype(np.float32)
    else:
        s = synth.scene_frame(width=8, height=8, n_lights=n, seed=101)
        pos, inten = s.light_pos.copy(), s.intensity.copy()
    if case == "duplicates":
        pos = np.repeat(pos[:2500], 8, axis=0)
    if case == "dark":
        inten[::2] = 0.0
    if case == "chain":  # intensities growing along the Morton order by 60 orders of magnitude
        t0 = oracle.Tree(pos, inten)
        inten = np.empty(n, np.float32)
        inten[t0.perm] = np.exp(np.linspace(-30, 30, n)).astype(np.float32)
    tree = ctx.build_light_tree(*_lights(pos, inten), topology="cost", cost_depth=depth)
    t = oracle.Tree(pos, inten, topology="cost", cost_depth=depth)
    _records_equal(tree, t)
    tree.free()


def test_cost_depth_is_checked(ctx):
    import paper_1907_12343_gb300 as hrr
    pos = synth.scene_frame(width=8, height=8, n_lights=100, seed=3).light_pos
    with pytest.raises(hrr.HRRError):
        ctx.build_light_tree(*_lights(pos, np.ones(100, np.float32)), topology="cost", cost_depth=65)


def test_culling_over_cost_trees_is_exact(ctx):
    s = synth.scene_frame(width=257, height=131, n_lights=50021, tile_w=64, tile_h=64, target=64.0, seed=7)
    g = upload_scene(s)
    ctx.set_shift_tile(s.tile)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology="cost")
    st, cnt, pairs, vis = run_cull(ctx, g, tree, float(s.tau), visits=True)
    assert st == 0
    t = oracle.Tree(s.light_pos, s.intensity, topology="cost")
    hier = oracle_hier(t, s.eye_pos, s.px, s.py, s.tile, s.tau)
    assert np.array_equal(sorted_pairs(pairs), sorted_pairs(hier["pairs"]))
    assert np.array_equal(vis, hier["visits"].astype(np.uint32))
    radix = oracle_hier(oracle.Tree(s.light_pos, s.intensity), s.eye_pos, s.px, s.py, s.tile, s.tau)
    assert hier["total_visits"] < radix["total_visits"]
    # refit keeps the cost topology
    jit = (synth.uniform01(5, 1, 3 * len(s.light_pos)).reshape(-1, 3) - 0.5) * 0.05
    pos = np.clip(s.light_pos + jit.astype(np.float32), 0, 1).astype(np.float32)
    ctx.refit_light_tree(tree, *_lights(pos, s.intensity))
    t.refit(pos, s.intensity)
    _records_equal(tree, t)
    tree.free()
