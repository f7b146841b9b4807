"""The node test is monotone along the hierarchy (the premise of the traversal's head).

A child's box lies inside its parent's, its maximum intensity is at most the parent's and
its range minimum (over a sub-range) at least the parent's, and the conservative cull test
of Sec. 1 (our division-free form, with directed rounding) culls at least as much for each.
So a parent's cull implies its children's, and a node below the root is visited by the
hierarchical traversal iff its own test passes. The GPU traversal's head evaluates the top
levels that way, without walking them; these tests check the property with the oracle's
own node test and range minimum against the oracle's traversal, per eye.
"""
import numpy as np

import oracle
import synth

F = np.float32


def _trees():
    rng = np.random.default_rng(17)
    out = []
    pos = rng.random((1500, 3)).astype(F)
    out.append(("uniform-radix", oracle.Tree(pos, np.exp(rng.normal(size=1500)).astype(F))))
    g = synth.gaussian_mixture_lights(1500, 8, seed=5)
    out.append(("gaussian-cost", oracle.Tree(g, np.exp(synth.normal(5, 2, 1500)).astype(F), topology="cost")))
    # lights at x = 2^-1 .. 2^-21 beside a cluster: leaves near the root
    x = (2.0 ** -np.arange(1, 22, dtype=np.float64)).astype(F)
    line = np.stack([x, np.full_like(x, 0.5), np.full_like(x, 0.5)], axis=1)
    lp = np.concatenate([line, (rng.random((600, 3)) * 1e-3).astype(F)]).astype(F)
    out.append(("line-radix", oracle.Tree(lp, np.ones(len(lp), F))))
    # 60 binary decades of intensity with the cost-driven splits
    cp = rng.random((1200, 3)).astype(F)
    out.append(("chain-cost", oracle.Tree(cp, (F(2.0) ** (-(np.arange(1200) % 60))).astype(F), topology="cost")))
    return out


def _own_culls(t, tau, e, r):
    """Per internal node: does its own test cull it (its box, maximum intensity and the
    range minimum over its leaf range, for an eye at e with shift r)?"""
    out = np.zeros(t.n - 1, bool)
    for g in range(t.n - 1):
        v, _ = oracle.rangemin_trie(int(t.first[g]), int(t.last[g]) + 1, int(r))
        out[g] = oracle.node_culls(tau, t.lo[g], t.hi[g], t.imax[g], e, v)
    return out


def _children(t, g):
    s = int(t.split[g])
    kids = []
    if int(t.first[g]) != s:
        kids.append(s)
    if s + 1 != int(t.last[g]):
        kids.append(s + 1)
    return kids


def test_visited_iff_own_test_passes():
    tile = synth.shift_tile(8, 8, 3)
    rng = np.random.default_rng(23)
    for name, t in _trees():
        eyes = rng.random((12, 3)).astype(F)
        px = np.arange(12, dtype=np.uint16) % 8
        py = np.arange(12, dtype=np.uint16) // 8
        for tau in (F(1e-4), F(3e-3)):
            hier = oracle.cull_hier(t, eyes, px, py, tile, tau, width=2)
            for j in range(len(eyes)):
                r = int(np.asarray(tile).reshape(-1)[int(py[j]) * 8 + int(px[j])])
                culls = _own_culls(t, tau, eyes[j], r)
                # a parent's cull implies its children's
                for g in range(t.n - 1):
                    if culls[g]:
                        assert all(culls[c] for c in _children(t, g)), (name, j, g)
                # the root always, and every other internal node iff its own test passes
                own = 1 + int(np.count_nonzero(~culls[1:]))
                assert own == int(hier["visits"][j]), (name, float(tau), j, own, int(hier["visits"][j]))
