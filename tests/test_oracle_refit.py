"""Refitting the oracle hierarchy for moved lights (the per-frame update of a served light
set): the leaf order and topology stay, the boxes and maximum intensities follow the new
positions, and hierarchical culling over the refitted tree still equals flat culling."""
import numpy as np

import oracle
import synth


def _moved(s, seed, scale=0.05):
    jitter = (synth.uniform01(seed, 1, 3 * len(s.light_pos)).reshape(-1, 3) - 0.5) * scale
    pos = np.clip(s.light_pos + jitter.astype(np.float32), 0.0, 1.0).astype(np.float32)
    inten = (s.intensity * (0.5 + synth.uniform01(seed, 2, len(s.intensity)))).astype(np.float32)
    return pos, inten


def test_refit_with_the_same_lights_changes_nothing():
    s = synth.scene_uniform(n_lights=2000, seed=61)
    t = oracle.Tree(s.light_pos, s.intensity)
    lo, hi, im = t.lo.copy(), t.hi.copy(), t.imax.copy()
    t.refit(s.light_pos, s.intensity)
    assert np.array_equal(t.lo, lo) and np.array_equal(t.hi, hi) and np.array_equal(t.imax, im)


def test_refitted_boxes_are_the_tight_boxes_of_the_moved_leaves():
    s = synth.scene_frame(width=8, height=8, n_lights=3001, seed=62)
    t = oracle.Tree(s.light_pos, s.intensity)
    first, last, split, perm = t.first.copy(), t.last.copy(), t.split.copy(), t.perm.copy()
    pos, inten = _moved(s, 63)
    t.refit(pos, inten)
    assert np.array_equal(t.first, first) and np.array_equal(t.split, split) and np.array_equal(t.perm, perm)
    leaf_pos, leaf_i = pos[perm], inten[perm]
    rng = np.random.default_rng(0)
    for k in rng.choice(len(first), 200, replace=False):
        p = leaf_pos[first[k]:last[k] + 1]
        # every leaf of the range is inside, and every face is touched by one of them
        assert np.all(p >= t.lo[k]) and np.all(p <= t.hi[k])
        assert np.array_equal(p.min(axis=0), t.lo[k]) and np.array_equal(p.max(axis=0), t.hi[k])
        assert t.imax[k] == leaf_i[first[k]:last[k] + 1].max()


def test_culling_over_a_refitted_tree_equals_flat():
    s = synth.scene_frame(width=16, height=9, n_lights=4099, tile_w=16, tile_h=16, target=32.0, seed=64)
    t = oracle.Tree(s.light_pos, s.intensity)
    pos, inten = _moved(s, 65, scale=0.2)
    t.refit(pos, inten)
    flat = oracle.cull_flat(t, s.eye_pos, s.px, s.py, s.tile, s.tau)
    hier = oracle.cull_hier(t, s.eye_pos, s.px, s.py, s.tile, s.tau)
    assert len(flat["pairs"]) > 0
    assert np.array_equal(np.sort(flat["pairs"].view(np.uint64).ravel()), np.sort(hier["pairs"].view(np.uint64).ravel()))
    # the leaf order is the build's: a fresh build over the moved lights orders them anew
    fresh = oracle.Tree(pos, inten)
    assert not np.array_equal(fresh.perm, t.perm)
