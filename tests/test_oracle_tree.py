"""Pins for the oracle's Morton sort and radix-tree hierarchy (CPU only).

The hierarchy only needs each node to be a contiguous leaf range (Sec. 1); these tests pin
the oracle's particular tree, a binary radix tree over (Morton key, sorted position), by
its defining invariants and by brute force on small inputs.
"""
import numpy as np
import pytest

import oracle
import synth

F = np.float32
CELL = 2.0 ** -21


def test_morton_closed_forms():
    assert oracle.morton(0, 0, 0) == 0
    assert oracle.morton(CELL, 0, 0) == 4
    assert oracle.morton(0, CELL, 0) == 2
    assert oracle.morton(0, 0, CELL) == 1
    assert oracle.morton(0.5, 0, 0) == 1 << 62
    top = float(np.nextafter(F(1), F(0)))
    assert oracle.morton(top, top, top) == (1 << 63) - 1
    # outside the unit cube: clamped to the border cells
    xs = sum(1 << (3 * k + 2) for k in range(21))
    assert oracle.morton(1.5, -1.0, 0.0) == xs
    # cell index is floor(x * 2^21): just below a cell boundary stays in the lower cell
    below = float(np.nextafter(F(3 * CELL), F(0)))
    assert oracle.morton(below, 0, 0) == oracle.morton(2 * CELL, 0, 0)


def _bit_interleave(cx, cy, cz):
    s = ""
    for k in range(20, -1, -1):
        s += str((cx >> k) & 1) + str((cy >> k) & 1) + str((cz >> k) & 1)
    return int(s, 2)


def test_morton_matches_string_interleave():
    rng = np.random.default_rng(1)
    pts = rng.random((2000, 3)).astype(F)
    for x, y, z in pts:
        c = [min(int(np.floor(float(v) * 2 ** 21)), 2 ** 21 - 1) for v in (x, y, z)]
        assert oracle.morton(x, y, z) == _bit_interleave(*c)


def _check_tree(pos, inten):
    t = oracle.Tree(pos, inten)
    n = len(inten)
    # sorting: permutation, keys ascending, equal keys by original id
    assert sorted(t.perm.tolist()) == list(range(n))
    keys = np.array([oracle.morton(*pos[i]) for i in t.perm], dtype=np.uint64)
    assert np.array_equal(keys, t.key)
    order = sorted(range(n), key=lambda i: (oracle.morton(*pos[i]), i))
    assert t.perm.tolist() == order
    assert np.array_equal(t.pos, pos[t.perm]) and np.array_equal(t.inten, inten[t.perm])
    if n == 1:
        assert t.height == 0
        return t
    ni = n - 1
    # every internal id used once; the root covers everything; each id sits at one end of
    # its range; children (split, split+1) partition the parent
    assert (t.first != 0xFFFFFFFF).all()
    assert t.first[0] == 0 and t.last[0] == n - 1
    seen_leaf = np.zeros(n, dtype=int)
    seen_internal = np.zeros(ni, dtype=int)
    seen_internal[0] += 1
    depth = {0: 1}
    stack = [0]
    height = 1
    while stack:
        k = stack.pop()
        f, l, s = int(t.first[k]), int(t.last[k]), int(t.split[k])
        assert f <= s < l
        assert k in (f, l)

        # splitting bit: highest difference of the (key, position) concatenations
        def aug(i):
            return (int(t.key[i]) << 32) | i
        hb = (aug(f) ^ aug(l)).bit_length() - 1
        for i in range(f, l + 1):
            assert ((aug(i) >> hb) & 1) == (0 if i <= s else 1)
        for cf, cl, cid in ((f, s, s), (s + 1, l, s + 1)):
            if cf == cl:
                seen_leaf[cf] += 1
            else:
                seen_internal[cid] += 1
                assert t.first[cid] == cf and t.last[cid] == cl
                depth[cid] = depth[k] + 1
                height = max(height, depth[cid])
                stack.append(cid)
        # boxes are the exact bounds of the range; imax its largest intensity
        assert np.array_equal(t.lo[k], t.pos[f:l + 1].min(axis=0))
        assert np.array_equal(t.hi[k], t.pos[f:l + 1].max(axis=0))
        assert t.imax[k] == t.inten[f:l + 1].max()
    assert (seen_leaf == 1).all() and (seen_internal == 1).all()
    assert t.height == height <= 96
    return t


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 100, 1000])
def test_tree_invariants_uniform(n):
    rng = np.random.default_rng(n)
    pos = rng.random((n, 3)).astype(F)
    inten = np.exp(rng.standard_normal(n)).astype(F)
    _check_tree(pos, inten)


def test_tree_invariants_duplicate_keys():
    # lights on a coarse grid: many equal Morton keys, split by sorted position
    rng = np.random.default_rng(9)
    pos = (rng.integers(0, 3, (300, 3)) / 3.0).astype(F)
    inten = rng.random(300).astype(F)
    _check_tree(pos, inten)
    # all lights in one place
    pos = np.full((33, 3), 0.25, F)
    t = _check_tree(pos, np.ones(33, F))
    assert t.perm.tolist() == list(range(33))


def test_tree_invariants_gaussian_mixture():
    pos = synth.gaussian_mixture_lights(3000, 8, seed=4)
    inten = np.exp(1.5 * synth.normal(4, 5, 3000)).astype(F)
    _check_tree(pos, inten)
