"""The oracle's plain C99 build (no OpenMP) compiles and computes what the default build
computes (CPU only).

The OpenMP pragmas only distribute independent eyes, pairs and queries over threads, so
the single-threaded build must return the same range minima, the same accepted sets and
the same connection weights.
"""
import ctypes as C
import os

import numpy as np

import oracle
import synth


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def test_plain_build_matches_default(tmp_path):
    path = oracle.build(force=True, openmp=False, out=os.path.join(str(tmp_path), "liboracle_plain.so"))
    L = oracle.configure(C.CDLL(path))
    assert L.or_max_threads() == 1

    # range minima, every method (ranges of at most 4096 indices, so the scan is quick)
    a, b, r = synth.rangemin_queries(2000, seed=5)
    b = (a.astype(np.uint64) + np.minimum(b - a, 4096)).astype(np.uint32)
    for name, m in oracle.METHODS.items():
        v = np.empty(len(a), np.uint32)
        k = np.empty(len(a), np.uint32)
        L.or_rangemin_batch(_ptr(a), _ptr(b), _ptr(r), len(a), m, 32, _ptr(v), _ptr(k), 0)
        v_ref, k_ref = oracle.rangemin_batch(a, b, r, name)
        assert np.array_equal(v, v_ref) and np.array_equal(k, k_ref), name

    # flat culling of a small scene: the same accepted pairs
    s = synth.scene_uniform(n_lights=300, grid_w=8, grid_h=6, tile_w=8, tile_h=8, target=12.0, seed=3)
    t = oracle.Tree(s.light_pos, s.intensity)
    ref = oracle.cull_flat(t, s.eye_pos, s.px, s.py, s.tile, s.tau)
    eye = np.ascontiguousarray(s.eye_pos, np.float32)
    px = np.ascontiguousarray(s.px, np.uint16)
    py = np.ascontiguousarray(s.py, np.uint16)
    tile = np.ascontiguousarray(s.tile, np.uint32)
    pos = np.ascontiguousarray(s.light_pos, np.float32)
    inten = np.ascontiguousarray(s.intensity, np.float32)
    tp = L.or_tree_build(_ptr(pos), _ptr(inten), len(inten))
    res = L.or_cull_flat(tp, _ptr(eye), _ptr(px), _ptr(py), None, len(eye), _ptr(tile),
                         tile.shape[1], tile.shape[0], np.float32(s.tau), 0)
    n = int(res.contents.n_pairs)
    got = np.ctypeslib.as_array(res.contents.pairs, shape=(2 * n,)).reshape(n, 2).copy()
    L.or_cull_free(res)
    L.or_tree_free(tp)
    assert np.array_equal(got, ref["pairs"])

    # connection weights (the call that used to need OpenMP's thread-count setter)
    w = np.zeros(n, np.float32)
    vis = np.zeros(n, np.uint8)
    sums = np.zeros(len(eye), np.float64)
    pairs = np.ascontiguousarray(got, np.uint32)
    no_tris = np.zeros(9, np.float32)
    L.or_connect(_ptr(eye), len(eye), _ptr(pos), _ptr(inten), _ptr(pairs), n, np.float32(s.tau),
                 _ptr(no_tris), 0, _ptr(w), _ptr(vis), _ptr(sums), 2)
    ref_c = oracle.connect(s.eye_pos, s.light_pos, s.intensity, got, s.tau)
    assert np.array_equal(w, ref_c["weight"]) and np.array_equal(sums, ref_c["eye_sum"])
