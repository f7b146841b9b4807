"""The space-time shift option of Sec. 3 (psi(j, n) from a 3D tile of precomputed shifts):
the oracle's layer selection and the seeded 3D tile's stratification."""
import numpy as np

import oracle
import synth


def _scene():
    return synth.scene_uniform(n_lights=600, grid_w=8, grid_h=8, tile_w=8, tile_h=8, target=12.0, seed=41)


def test_layer_selection_wraps_modulo_depth():
    s = _scene()
    t3 = synth.shift_tile_3d(8, 8, 4, seed=42)
    tree = oracle.Tree(s.light_pos, s.intensity)
    res = [oracle.cull_flat(tree, s.eye_pos, s.px, s.py, t3, s.tau, sample_index=n)["pairs"] for n in range(6)]
    assert np.array_equal(res[0], res[4]) and np.array_equal(res[1], res[5])
    # different layers shift every pixel by a different stratum: different accepted sets
    assert not np.array_equal(res[0], res[1]) and not np.array_equal(res[1], res[2])


def test_constant_layers_equal_constant_plain_tiles():
    s = _scene()
    tree = oracle.Tree(s.light_pos, s.intensity)
    consts = np.array([0, 0x40000000, 0x9E3779B9], dtype=np.uint32)
    t3 = np.broadcast_to(consts[:, None, None], (3, 8, 8)).copy()
    for n in range(5):
        flat3 = oracle.cull_flat(tree, s.eye_pos, s.px, s.py, t3, s.tau, sample_index=n)
        flat2 = oracle.cull_flat(tree, s.eye_pos, s.px, s.py, np.full((8, 8), consts[n % 3], np.uint32), s.tau)
        assert np.array_equal(flat3["pairs"], flat2["pairs"])


def test_depth_one_is_the_plain_tile():
    s = _scene()
    tree = oracle.Tree(s.light_pos, s.intensity)
    a = oracle.cull_hier(tree, s.eye_pos, s.px, s.py, s.tile, s.tau)
    b = oracle.cull_hier(tree, s.eye_pos, s.px, s.py, s.tile[None], s.tau, sample_index=7)
    assert np.array_equal(a["pairs"], b["pairs"]) and np.array_equal(a["visits"], b["visits"])


def test_seeded_3d_tile_is_stratified_in_time_and_balanced_in_space():
    d = 8
    t3 = synth.shift_tile_3d(16, 16, d, seed=5)
    strata = (t3.astype(np.uint64) * d) >> np.uint64(32)
    # every pixel visits every stratum of [0, 1) once over the d samples
    assert np.all(np.sort(strata, axis=0) == np.arange(d, dtype=np.uint64)[:, None, None])
    # every layer holds each stratum equally often
    for layer in strata:
        assert np.all(np.bincount(layer.ravel().astype(np.int64), minlength=d) == 16 * 16 // d)
    # within a stratum, the fine part keeps the blue-noise rank order of the base tile
    base = synth.void_and_cluster(16, 16, 5)
    fine = (t3[0].astype(np.uint64) * d) & np.uint64(0xFFFFFFFF)
    assert np.array_equal(np.argsort(fine.ravel(), kind="stable"), np.argsort(base.ravel(), kind="stable"))
    # depth 1 reduces to a plain tile of the base ranks
    t1 = synth.shift_tile_3d(16, 16, 1, seed=5)[0]
    assert np.array_equal(np.argsort(t1.ravel(), kind="stable"), np.argsort(base.ravel(), kind="stable"))
