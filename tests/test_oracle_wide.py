"""Pins for the oracle's traversal with nodes of width four (CPU only).

Sec. 1 needs only a hierarchy of contiguous leaf ranges; reading the binary tree with
nodes of width four (a visit tests the grandchildren) must keep the accepted set (equal
to the flat brute force) and visit exactly the even-depth nodes that the binary traversal
visits, because the cull test is monotone: a box inside another, a smaller maximum
intensity and a range minimum over a sub-range never turn a cull into a visit.
"""
import numpy as np
import pytest

import oracle
import synth

F = np.float32


def _scenes():
    out = [("uniform", dict(synth.scene_uniform()), "radix")]
    out.append(("frame", dict(synth.scene_frame(width=61, height=37, n_lights=5003, tile_w=16, tile_h=16,
                                                 target=48.0, seed=5)), "cost"))
    for n in (1, 2, 3, 4, 5, 31):
        s = dict(synth.scene_uniform(n_lights=max(n, 2), grid_w=8, grid_h=8, tile_w=8, tile_h=8,
                                     target=1.0, seed=6))
        s["light_pos"], s["intensity"] = s["light_pos"][:n], s["intensity"][:n]
        s["tau"] = F(s["tau"] * 3)
        out.append((f"tiny{n}", s, "radix"))
    dup = dict(synth.scene_uniform(n_lights=400, grid_w=8, grid_h=8, tile_w=8, tile_h=8, seed=11))
    dup["light_pos"] = np.repeat(dup["light_pos"][:50], 8, axis=0)
    out.append(("duplicates", dup, "cost"))
    return out


@pytest.mark.parametrize("name,scene,topology", _scenes(), ids=[x[0] for x in _scenes()])
def test_wide_traversal_equals_flat(name, scene, topology):
    t = oracle.Tree(scene["light_pos"], scene["intensity"], topology=topology)
    args = (t, scene["eye_pos"], scene["px"], scene["py"], scene["tile"], scene["tau"])
    flat = oracle.cull_flat(*args)
    h2 = oracle.cull_hier(*args)
    h4 = oracle.cull_hier(*args, width=4)
    assert np.array_equal(flat["pairs"], h4["pairs"])
    assert np.array_equal(flat["count"], h4["count"])
    if t.n > 2:
        assert h4["total_visits"] < h2["total_visits"]


def _binary_visited(t, e, r, tau):
    """Python restatement of the binary traversal: the set of visited internal nodes."""
    seen, stack = set(), [0]
    while stack:
        g = stack.pop()
        seen.add(g)
        s = int(t.split[g])
        for f, l, k in ((int(t.first[g]), s, s), (s + 1, int(t.last[g]), s + 1)):
            if f == l:
                continue
            v, _ = oracle.rangemin_trie(f, l + 1, r)
            if not oracle.node_culls(tau, t.lo[k], t.hi[k], t.imax[k], e, v):
                stack.append(k)
    return seen


def _depths(t):
    d = {0: 0}
    order = [0]
    for g in order:
        s = int(t.split[g])
        for f, l, k in ((int(t.first[g]), s, s), (s + 1, int(t.last[g]), s + 1)):
            if f != l:
                d[k] = d[g] + 1
                order.append(k)
    return d


def test_wide_visits_are_the_even_depth_binary_visits():
    s = synth.scene_frame(width=24, height=16, n_lights=2500, tile_w=16, tile_h=16, target=40.0, seed=13)
    for topology in ("radix", "cost"):
        t = oracle.Tree(s["light_pos"], s["intensity"], topology=topology)
        depth = _depths(t)
        h4 = oracle.cull_hier(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"], width=4)
        h2 = oracle.cull_hier(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"])
        for j in range(0, len(s["eye_pos"]), 7):
            r = int(s["tile"][int(s["py"][j]) % 16, int(s["px"][j]) % 16])
            seen = _binary_visited(t, s["eye_pos"][j], r, s["tau"])
            assert len(seen) == int(h2["visits"][j])
            assert sum(1 for g in seen if depth[g] % 2 == 0) == int(h4["visits"][j])


def test_cull_test_is_monotone_under_nesting():
    # the property the wide traversal rests on, checked on random nested boxes
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(4000):
        e = rng.random(3).astype(F)
        lo = rng.random(3).astype(F)
        hi = (lo + rng.random(3) * 0.3).astype(F)
        ilo = (lo + (hi - lo) * rng.random(3) * 0.5).astype(F)
        ihi = np.minimum(hi, ilo + (hi - ilo) * rng.random(3)).astype(F)
        ihi = np.maximum(ihi, ilo)
        imax = F(np.exp(rng.normal()))
        imin = F(imax * rng.random())
        tau = F(10 ** rng.uniform(-7, -3))
        v = int(rng.integers(1, 2 ** 32))
        v_in = min(2 ** 32 - 1, v + int(rng.integers(0, 2 ** 28)))
        if oracle.node_culls(tau, lo, hi, imax, e, v):
            checked += 1
            assert oracle.node_culls(tau, ilo, ihi, imin, e, v_in)
    assert checked > 200
