"""Pins for the oracle's flat and hierarchical culling (CPU only).

* Closed forms from the stratification of Phi_2: lights sitting on the eye with a dyadic
  acceptance probability accept exactly a residue class of sorted positions; for 2^k
  lights any shift and any probability accept within one of 2^k p.
* The paper's claim that the hierarchy only removes work (Sec. 1): the hierarchical set
  equals the flat brute-force set on several scenes and corner cases.
* Statistical sanity: accepted counts per eye track the expected count sum_i p_ij.
"""
import numpy as np
import pytest

import oracle
import synth

F = np.float32


def _pairs_set(res):
    return set(map(tuple, res["pairs"].tolist()))


def _one_eye(n, tau, shift):
    pos = np.full((n, 3), 0.5, F)
    eye = np.full((1, 3), 0.5, F)
    px = py = np.zeros(1, np.uint16)
    tile = np.array([[shift]], np.uint32)
    return oracle.Tree(pos, np.ones(n, F)), eye, px, py, tile, F(tau)


@pytest.mark.parametrize("fn", [oracle.cull_flat, oracle.cull_hier])
def test_dyadic_probability_selects_residue_class(fn):
    # p = 1/2 with r = 0 accepts brev(i) < 2^31, i.e. every even sorted position; r = 2^31
    # accepts the odd ones; p = 1/4 with r = 0 accepts i = 0 mod 4.
    n = 100
    md = F(1e-4)
    t, eye, px, py, tile, tau = _one_eye(n, F(0.5) * md, 0)
    assert fn(t, eye, px, py, tile, tau)["pairs"][:, 1].tolist() == list(range(0, n, 2))
    t, eye, px, py, tile, tau = _one_eye(n, F(0.5) * md, 1 << 31)
    assert fn(t, eye, px, py, tile, tau)["pairs"][:, 1].tolist() == list(range(1, n, 2))
    t, eye, px, py, tile, tau = _one_eye(n, F(0.25) * md, 0)
    assert fn(t, eye, px, py, tile, tau)["pairs"][:, 1].tolist() == list(range(0, n, 4))


@pytest.mark.parametrize("k", [4, 7, 10])
def test_stratified_count_within_one(k):
    # for 2^k lights the values brev(i) are the multiples of 2^(32-k); any rotation puts
    # floor or ceil of 2^k * t / 2^32 of them below a threshold t
    n = 1 << k
    md = F(1e-4)
    rng = np.random.default_rng(k)
    for _ in range(20):
        p = F(rng.random())
        shift = int(rng.integers(0, 2 ** 32))
        t, eye, px, py, tile, tau = _one_eye(n, p * md, shift)
        res = oracle.cull_hier(t, eye, px, py, tile, tau)
        thr = oracle.leaf_threshold(tau, eye[0], F(1), eye[0])
        expect = n * thr / 2 ** 32
        assert abs(int(res["count"][0]) - expect) <= 1.0
        assert _pairs_set(res) == _pairs_set(oracle.cull_flat(t, eye, px, py, tile, tau))


def _hier_equals_flat(scene, eye_ids=None):
    t = oracle.Tree(scene["light_pos"], scene["intensity"])
    args = (t, scene["eye_pos"], scene["px"], scene["py"], scene["tile"], scene["tau"])
    flat = oracle.cull_flat(*args, eye_ids=eye_ids)
    hier = oracle.cull_hier(*args, eye_ids=eye_ids)
    assert np.array_equal(flat["pairs"], hier["pairs"])
    assert np.array_equal(flat["count"], hier["count"])
    return t, flat, hier


def test_hier_equals_flat_uniform_scene():
    s = synth.scene_uniform()
    t, flat, hier = _hier_equals_flat(s)
    mean = flat["count"].mean()
    assert 20 < mean < 45, mean  # tau calibrated for about 32 accepted per eye
    # the hierarchy visits far fewer internal nodes than the flat loop tests pairs
    assert hier["total_visits"] < 0.25 * len(s["eye_pos"]) * t.n


def test_hier_equals_flat_small_frame():
    s = synth.scene_frame(width=61, height=37, n_lights=5003, tile_w=16, tile_h=16,
                          target=48.0, seed=5)
    _hier_equals_flat(s)


@pytest.mark.parametrize("n_lights", [1, 2, 3, 4, 31])
def test_hier_equals_flat_tiny_light_sets(n_lights):
    s = dict(synth.scene_uniform(n_lights=max(n_lights, 2), grid_w=8, grid_h=8, tile_w=8,
                                 tile_h=8, target=1.0, seed=6))
    s["light_pos"] = s["light_pos"][:n_lights]
    s["intensity"] = s["intensity"][:n_lights]
    s["tau"] = F(s["tau"] * 3)
    _hier_equals_flat(s)


def test_all_or_nothing():
    s = dict(synth.scene_uniform(n_lights=300, grid_w=8, grid_h=4, tile_w=8, tile_h=8, seed=7))
    t = oracle.Tree(s["light_pos"], s["intensity"])
    base = (t, s["eye_pos"], s["px"], s["py"], s["tile"])
    assert oracle.cull_hier(*base, F(0))["pairs"].shape[0] == 0
    everything = oracle.cull_hier(*base, F(1e30))
    assert everything["pairs"].shape[0] == 32 * 300
    assert _pairs_set(everything) == {(j, i) for j in range(32) for i in range(300)}


def test_eye_ids_label_output():
    s = synth.scene_uniform(n_lights=500, grid_w=8, grid_h=8, tile_w=8, tile_h=8, seed=8)
    t = oracle.Tree(s["light_pos"], s["intensity"])
    ids = np.arange(64, dtype=np.uint32)[::3]
    sub = oracle.cull_hier(t, s["eye_pos"][ids], s["px"][ids], s["py"][ids], s["tile"], s["tau"],
                           eye_ids=ids)
    full = oracle.cull_hier(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"])
    keep = np.isin(full["pairs"][:, 0], ids)
    assert np.array_equal(sub["pairs"], full["pairs"][keep])


def test_counts_track_expected_acceptance():
    # each eye's accepted count has mean sum_i p_ij; with the stratified sequence the
    # deviation should not exceed what independent Bernoulli draws would give
    s = synth.scene_uniform()
    t = oracle.Tree(s["light_pos"], s["intensity"])
    res = oracle.cull_flat(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"])
    lp = s["light_pos"].astype(np.float64)
    li = s["intensity"].astype(np.float64)
    dev, sd = [], []
    for j in range(0, len(s["eye_pos"]), 8):
        d2 = ((lp - s["eye_pos"][j].astype(np.float64)) ** 2).sum(axis=1)
        p = np.minimum(1.0, float(s["tau"]) * li / np.maximum(d2, 1e-4))
        dev.append(abs(int(res["count"][j]) - p.sum()))
        sd.append(np.sqrt((p * (1 - p)).sum()))
    assert np.mean(dev) < np.mean(sd)
