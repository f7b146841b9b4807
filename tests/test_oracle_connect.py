"""Connection evaluation in the oracle (the step after the culling): the Russian-roulette
weight of an accepted connection, and segment-triangle visibility (Moller-Trumbore in
float32), pinned to closed forms, an independent float64 solve and the estimator's
unbiasedness."""
import numpy as np

import oracle
import synth

TRI = np.array([0, 0, 0.5, 1, 0, 0.5, 0, 1, 0.5], np.float32)  # right triangle in z = 0.5


def test_segment_closed_forms():
    assert oracle.segment_hits([0.2, 0.2, 0.0], [0.2, 0.2, 1.0], TRI)          # t = 0.5, inside
    assert not oracle.segment_hits([0.2, 0.2, 0.0], [0.2, 0.2, 0.4], TRI)      # ends before the plane
    assert not oracle.segment_hits([0.2, 0.2, 0.6], [0.2, 0.2, 1.0], TRI)      # starts after it
    assert not oracle.segment_hits([0.0, 0.2, 0.5], [1.0, 0.3, 0.5], TRI)      # in the plane: det = 0
    assert not oracle.segment_hits([0.6, 0.6, 0.0], [0.6, 0.6, 1.0], TRI)      # u + v = 1.2 > 1
    assert not oracle.segment_hits([-0.1, 0.2, 0.0], [-0.1, 0.2, 1.0], TRI)    # u < 0
    assert oracle.segment_hits([0.2, 0.2, 1.0], [0.2, 0.2, 0.0], TRI)          # either direction
    # the plane at t = 0.00005 and t = 0.99995 is outside the open range (1e-4, 1 - 1e-4)
    assert not oracle.segment_hits([0.2, 0.2, 0.49995], [0.2, 0.2, 1.49995], TRI)
    assert not oracle.segment_hits([0.2, 0.2, -0.49995], [0.2, 0.2, 0.50005], TRI)


def test_segment_against_a_float64_solve():
    rng = np.random.default_rng(7)
    agree = checked = 0
    for _ in range(4000):
        v = rng.random((3, 3))
        e, l = rng.random(3), rng.random(3)
        # e + t (l - e) = v0 + u (v1 - v0) + w (v2 - v0)
        A = np.stack([l - e, v[0] - v[1], v[0] - v[2]], axis=1)
        if abs(np.linalg.det(A)) < 1e-3:
            continue
        t, u, w = np.linalg.solve(A, v[0] - e)
        margin = min(t - 1e-4, 1 - 1e-4 - t, u, w, 1 - u - w)
        if abs(margin) < 1e-3:
            continue  # too close to an edge or an end for float32 to be decisive
        want = margin > 0
        got = oracle.segment_hits(e.astype(np.float32), l.astype(np.float32), v.astype(np.float32))
        checked += 1
        agree += got == want
        # winding does not matter
        assert oracle.segment_hits(e.astype(np.float32), l.astype(np.float32), v[[0, 2, 1]].astype(np.float32)) == got
    assert checked > 2000 and agree == checked


def test_weight_closed_forms():
    # dyadic coordinates: d^2 = 1/8, tau I = 1/32, p = 1/4 exactly
    e = np.array([0.25, 0.5, 0.375], np.float32)
    l = np.array([0.5, 0.75, 0.375], np.float32)
    w, p = oracle.pair_weight(2.0 ** -6, l, 2.0, e)
    assert p == 0.25 and w == 64.0  # p < 1: (I / d^2) / (tau I / d^2) = 1 / tau
    w1, p1 = oracle.pair_weight(100.0, l, 2.0, e)  # p clamps to 1: the weight is I / d^2
    assert p1 == 1.0 and w1 == 16.0
    w2, _ = oracle.pair_weight(100.0, e, 2.0, e)   # coincident: d^2 floors at 1e-4
    assert w2 == np.float32(2.0) / np.float32(1e-4)
    # away from dyadic values the weight is 1 / tau up to the float32 roundings of p
    rng = np.random.default_rng(3)
    for _ in range(200):
        e, l = rng.random(3).astype(np.float32), rng.random(3).astype(np.float32)
        w, p = oracle.pair_weight(1e-4, l, 1.0, e)
        if p < 1:
            assert abs(w * 1e-4 - 1) < 4e-7


def test_estimator_is_unbiased_over_random_shifts():
    # E over the shift r of the sum over accepted lights of I / d^2 / p equals the sum over
    # all lights of I / d^2: Russian roulette with the QMC sequence keeps it unbiased.
    s = synth.scene_frame(width=4, height=2, n_lights=2048, tile_w=4, tile_h=2, target=16.0, seed=9)
    tree = oracle.Tree(s.light_pos, s.intensity)
    exact = np.zeros(len(s.eye_pos))
    for j, e in enumerate(s.eye_pos.astype(np.float64)):
        d2 = np.maximum(((s.light_pos.astype(np.float64) - e) ** 2).sum(1), 1e-4)
        exact[j] = (s.intensity / d2).sum()
    n_samples = 600
    shifts = (synth.splitmix64(11, 3, n_samples) >> np.uint64(32)).astype(np.uint32)
    est = np.zeros((n_samples, len(s.eye_pos)))
    for k, r in enumerate(shifts):
        tile = np.full(s.tile.shape, r, np.uint32)
        fl = oracle.cull_flat(tree, s.eye_pos, s.px, s.py, tile, s.tau)
        est[k] = oracle.connect(s.eye_pos, s.light_pos, s.intensity, fl["pairs"], s.tau)["eye_sum"]
    mean, se = est.mean(0), est.std(0) / np.sqrt(n_samples)
    assert np.all(np.abs(mean - exact) < 5 * se + 1e-6 * exact)
    assert np.all(se < 0.05 * exact)  # the test has power: 5 standard errors are < 25%


def test_connect_visibility_and_sums():
    s = synth.scene_frame(width=8, height=4, n_lights=1500, tile_w=8, tile_h=4, target=24.0, seed=12)
    tree = oracle.Tree(s.light_pos, s.intensity)
    fl = oracle.cull_flat(tree, s.eye_pos, s.px, s.py, s.tile, s.tau)
    none = oracle.connect(s.eye_pos, s.light_pos, s.intensity, fl["pairs"], s.tau)
    assert none["visible"].all()
    tris = synth.occluder_triangles(4000, 13, size=0.02)
    occ = oracle.connect(s.eye_pos, s.light_pos, s.intensity, fl["pairs"], s.tau, tris)
    assert 0.05 < occ["visible"].mean() < 0.95
    assert np.array_equal(occ["weight"], np.where(occ["visible"], none["weight"], 0.0).astype(np.float32))
    for k in np.flatnonzero(~occ["visible"])[:50]:
        j, i = fl["pairs"][k]
        assert any(oracle.segment_hits(s.eye_pos[j], s.light_pos[i], t) for t in tris)
    want = np.zeros(len(s.eye_pos))
    np.add.at(want, fl["pairs"][:, 0], occ["weight"].astype(np.float64))
    assert np.allclose(occ["eye_sum"], want, rtol=1e-12)
