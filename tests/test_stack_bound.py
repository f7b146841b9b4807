"""The traversal's stack bound, checked by simulation on the CPU.

The culling kernel walks each eye's hierarchy with one warp: every step pops the newest
min(32, S) pending nodes (one per lane), and each lane pushes the surviving children of
its node (at most 2 for binary records, at most 4 for 4-wide records) as one run on top
of the stack. Its global-memory spill area is sized by the bound

    S <= (w - 1) * 32 * L + 32,

where w is the node width and L the number of depth levels at which a pushed node can
sit (binary: depths 1 .. H-1 of a tree of height H, so L = H - 1; 4-wide: the even
depths 2, 4, .. <= H - 1, so L = floor((H - 1) / 2)).

Why it holds: a run pushed in one step has at most 32 w entries; the next step, which
finds it on top, pops 32 of them or all of them, so whatever remains of a run below the
top holds at most (w - 1) 32 entries. Everything above a remainder descends (strictly)
from entries of that remainder's run, so the shallowest depth of the runs with
remainders increases strictly from the bottom of the stack to its top: at most L - 1
remainders lie below a top run of at most 32 w entries, or L remainders with no top run.

These tests replay the kernel's stack discipline on oracle trees of several shapes, for
any survive decisions (all children kept, which is the deepest stack, and seeded random
choices), and check the bound the kernel allocates for.
"""
import numpy as np
import pytest

import oracle
import synth

F = np.float32


def _children(t, g):
    """Internal children (binary ids) and leaf count of binary internal node g."""
    s = int(t.split[g])
    f, l = int(t.first[g]), int(t.last[g])
    out = []
    if f != s:
        out.append(s)
    if s + 1 != l:
        out.append(s + 1)
    return out


def _depths(t):
    d = np.zeros(t.n - 1, np.int64)
    order = [0]
    for g in order:
        for c in _children(t, g):
            d[c] = d[g] + 1
            order.append(c)
    return d


def _head_frontier(t, keep, levels=6):
    """The stack a binary walk with the head starts from: the nodes of depth levels - 1
    that survive, in heap (left to right) order, with the visits the head accounts for (the
    root and the surviving nodes above that depth). A node below the root survives iff
    keep(node) holds for it and every ancestor below the root, as for the walk itself."""
    front, visits = [0], 1
    for depth in range(1, levels):
        nxt = [c for g in front for c in _children(t, g) if keep(c)]
        if depth < levels - 1:
            visits += len(nxt)
        front = nxt
    return front, visits


def simulate(t, width, keep, lanes=32, head=False):
    """Largest stack size of the chunked traversal; keep(node) decides whether a pushed
    candidate survives its cull test. With head (binary only), the walk starts from the
    head's frontier at depth 5. Returns (max size, visits)."""
    stack = [0]
    peak, visits = 1, 0
    if head:
        stack, visits = _head_frontier(t, keep)
        peak = len(stack)
    while stack:
        m = min(lanes, len(stack))
        popped = stack[len(stack) - m:]
        del stack[len(stack) - m:]
        visits += m
        run = []
        for g in popped:
            if width == 2:
                cand = _children(t, g)
            else:
                cand = [gc for c in _children(t, g) for gc in _children(t, c)]
            run.extend(c for c in cand if keep(c))
        stack.extend(run)
        peak = max(peak, len(stack))
    return peak, visits


def bound(height, width, lanes=32):
    levels = height - 1 if width == 2 else (height - 1) // 2
    return (width - 1) * lanes * max(levels, 0) + lanes


def _trees():
    rng = np.random.default_rng(7)
    out = []
    # uniform cube, Gaussian clusters, a line of lights (deep radix trees) and an
    # exponential chain of intensities with the cost-driven splits (deep cost trees)
    pos = rng.random((3000, 3)).astype(F)
    out.append(("uniform", oracle.Tree(pos, np.ones(3000, F))))
    g = synth.gaussian_mixture_lights(4000, 8, seed=3)
    gp = g[0] if isinstance(g, tuple) else g
    out.append(("gaussian-cost", oracle.Tree(gp, np.ones(len(gp), F), topology="cost")))
    x = (2.0 ** -np.arange(1, 22, dtype=np.float64)).astype(F)
    line = np.stack([x, np.zeros_like(x), np.zeros_like(x)], axis=1)
    line = np.concatenate([line, rng.random((500, 3)).astype(F) * F(1e-6)], axis=0)
    out.append(("line", oracle.Tree(line, np.ones(len(line), F))))
    chain = rng.random((2000, 3)).astype(F)
    out.append(("chain-cost", oracle.Tree(chain, (F(2.0) ** (-np.arange(2000) % 60)).astype(F),
                                          topology="cost")))
    return out


def test_stack_bound_holds_from_the_head():
    # the head (binary records) starts the walk from at most 32 nodes of depth 5, one run
    # of the proof's kind; the bound and the visit count are those of the walk from the root
    for name, t in _trees():
        b = bound(int(t.height), 2)
        for p in (1.0, 0.5, 0.8, 0.95):
            seed = int(p * 1000) + 7
            h = lambda c, seed=seed: ((c * 0x9E3779B1 + seed * 0x85EBCA6B) & 0xFFFFFFFF) / 2.0 ** 32
            keep = (lambda c: True) if p == 1.0 else (lambda c, h=h, p=p: h(c) < p)
            peak, v = simulate(t, 2, keep, head=True)
            assert peak <= b, (name, p, peak, b)
            assert v == simulate(t, 2, keep)[1], (name, p)


@pytest.mark.parametrize("width", [2, 4])
def test_stack_bound_holds(width):
    for name, t in _trees():
        H = int(t.height)
        assert H >= 1, name
        b = bound(H, width)
        full, v = simulate(t, width, lambda c: True)
        assert full <= b, (name, width, full, b)
        for p in (0.5, 0.8, 0.95):
            seed = int(p * 1000) + width
            h = lambda c, seed=seed: ((c * 0x9E3779B1 + seed * 0x85EBCA6B) & 0xFFFFFFFF) / 2.0 ** 32
            peak, _ = simulate(t, width, lambda c, h=h, p=p: h(c) < p)
            assert peak <= b, (name, width, p, peak, b)


def test_bound_is_not_loose_by_much():
    # A perfectly balanced full traversal reaches a large part of the bound: the bound
    # is the right order, and the kernel's spill area (sized by it) is not wasted.
    n = 1 << 12
    pos = np.zeros((n, 3), F)
    cells = np.arange(n)
    pos[:, 0] = (cells.astype(np.float64) / n).astype(F)
    t = oracle.Tree(pos, np.ones(n, F))
    H = int(t.height)
    assert H == 12
    peak, visits = simulate(t, 2, lambda c: True)
    assert visits == n - 1
    assert bound(H, 2) // 4 <= peak <= bound(H, 2)
    depth = _depths(t)
    assert int(depth.max()) == H - 1
