"""Cost-driven splits over the Morton leaf order (the hierarchy the benchmark builds): the
oracle's rule against closed forms, a float64 restatement of the rule, tree validity, the
height bound, and hierarchical culling equal to flat culling (the leaf order, and so the
accepted set, are the radix tree's)."""
import numpy as np
import pytest

import oracle
import synth


def _check_tree(t):
    n = t.n
    if n == 1:
        return
    seen = np.zeros(n, int)
    stack = [0]
    while stack:
        k = stack.pop()
        f, l, s = int(t.first[k]), int(t.last[k]), int(t.split[k])
        assert f <= s < l and k in (f, l)
        for cf, cl, cid in ((f, s, s), (s + 1, l, s + 1)):
            if cf == cl:
                seen[cf] += 1
            else:
                assert t.first[cid] == cf and t.last[cid] == cl
                stack.append(cid)
    assert np.all(seen == 1)
    assert t.height <= 48 + 96


def test_dark_lights_split_in_the_middle():
    # zero intensities: every candidate costs exactly 0, ties go to the middle, so the tree
    # is perfectly balanced
    for n in (8, 16, 64, 2048):
        rng = np.random.default_rng(n)
        pos = rng.random((n, 3)).astype(np.float32)
        t = oracle.Tree(pos, np.zeros(n, np.float32), topology="cost")
        _check_tree(t)
        assert t.height == int(np.log2(n))
        assert t.split[0] == n // 2 - 1


def test_two_clusters_are_separated_at_the_root():
    rng = np.random.default_rng(1)
    a = (0.1 + 0.01 * rng.random((300, 3))).astype(np.float32)
    b = (0.8 + 0.01 * rng.random((200, 3))).astype(np.float32)
    t = oracle.Tree(np.concatenate([a, b]), np.ones(500, np.float32), topology="cost")
    _check_tree(t)
    left = set(t.perm[: int(t.split[0]) + 1].tolist())
    assert left == set(range(300))


def _rule(pos, inten, f, l):
    """The split rule restated in float32 numpy (every operation rounded to float32): every
    split, the child cost u^2 ((A + 0.1 P) + 1e-4) c sqrt(c) with u the child's maximum over
    the range's, ties."""
    f32 = np.float32
    P = pos[f:l + 1].astype(f32)
    I = inten[f:l + 1].astype(f32)

    def child(m, inv, d, c):
        u = m * inv
        a = (d[0] * d[1] + d[1] * d[2]) + d[2] * d[0]
        per = (d[0] + d[1]) + d[2]
        g = (a + f32(0.1) * per) + f32(1e-4)
        c = f32(c)
        return ((u * u) * g) * (c * np.sqrt(c))

    best = None
    for k in range(f, l):
        L, R = P[: k - f + 1], P[k - f + 1:]
        ml, mr = max(I[: k - f + 1].max(), f32(0)), max(I[k - f + 1:].max(), f32(0))
        mx = max(ml, mr)
        inv = f32(1) / max(mx, f32(np.finfo(f32).tiny)) if mx > 0 else f32(0)
        cl, cr = k - f + 1, l - k
        cost = child(ml, inv, L.max(0) - L.min(0), cl) + child(mr, inv, R.max(0) - R.min(0), cr)
        assert cost.dtype == f32
        key = (float(cost), abs(cl - cr), k)
        best = key if best is None or key < best else best
    return best[2]


@pytest.mark.parametrize("n,seed", [(2, 1), (3, 2), (40, 3), (1000, 4), (5000, 5)])
def test_splits_follow_the_rule(n, seed):
    s = synth.scene_frame(width=8, height=8, n_lights=n, seed=seed)
    t = oracle.Tree(s.light_pos, s.intensity, topology="cost")
    _check_tree(t)
    ks = [0] + [k for k in range(1, n - 1) if t.first[k] != t.last[k]][:6]
    for k in ks:
        f, l = int(t.first[k]), int(t.last[k])
        if l - f + 1 > 1 and (k == 0 or l - f < 3000):
            assert t.split[k] == _rule(t.pos, t.inten, f, l)


@pytest.mark.parametrize("case", ["uniform", "mixture", "duplicates", "zero", "tiny", "chain"])
def test_hierarchical_culling_equals_flat(case):
    if case == "uniform":
        s = dict(synth.scene_uniform(n_lights=3000, seed=91))
    else:
        s = dict(synth.scene_frame(width=24, height=16, n_lights=4001, tile_w=16, tile_h=16, target=24.0, seed=92))
    if case == "duplicates":
        s["light_pos"] = np.repeat(s["light_pos"][:500], 8, axis=0)[:4001]
    if case == "zero":
        s["intensity"] = np.where(np.arange(4001) % 3 == 0, 0.0, s["intensity"]).astype(np.float32)
    if case == "tiny":
        s["light_pos"], s["intensity"] = s["light_pos"][:17], s["intensity"][:17] * 50
    if case == "chain":  # intensities that grow along the Morton order push the cost rule to chains
        t0 = oracle.Tree(s["light_pos"], s["intensity"])
        inten = np.empty(len(s["intensity"]), np.float32)
        inten[t0.perm] = np.exp(np.linspace(-20, 20, len(inten))).astype(np.float32)
        s["intensity"] = inten
    t = oracle.Tree(s["light_pos"], s["intensity"], topology="cost")
    _check_tree(t)
    flat = oracle.cull_flat(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"])
    hier = oracle.cull_hier(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"])
    key = lambda p: np.sort(p.astype(np.uint64)[:, 0] << np.uint64(32) | p.astype(np.uint64)[:, 1])
    assert np.array_equal(key(flat["pairs"]), key(hier["pairs"]))
    radix = oracle.Tree(s["light_pos"], s["intensity"])
    assert np.array_equal(radix.perm, t.perm)


def test_fewer_visits_than_the_radix_tree_on_the_frame_workload():
    s = synth.scene_frame(width=48, height=27, n_lights=1 << 15, tile_w=16, tile_h=16, target=48.0, seed=93)
    v = {}
    for topo in ("radix", "cost"):
        t = oracle.Tree(s.light_pos, s.intensity, topology=topo)
        v[topo] = oracle.cull_hier(t, s.eye_pos, s.px, s.py, s.tile, s.tau)["total_visits"]
    assert v["cost"] < 0.92 * v["radix"]


def _radix_rule(keys, f, l):
    """The radix split restated: the last k whose key has a 0 at the highest bit where the
    keys of f and l differ; for equal keys, the same on the positions f and l."""
    kf, kl = int(keys[f]), int(keys[l])
    if kf != kl:
        bit = (kf ^ kl).bit_length() - 1
        digits = [(int(keys[k]) >> bit) & 1 for k in range(f, l + 1)]
    else:
        bit = (f ^ l).bit_length() - 1
        digits = [(k >> bit) & 1 for k in range(f, l + 1)]
    return f + max(i for i, d in enumerate(digits) if d == 0)


@pytest.mark.parametrize("depth", [1, 3, 6])
def test_cost_depth_hands_over_to_radix_splits(depth):
    s = synth.scene_frame(width=8, height=8, n_lights=1500, seed=11)
    t = oracle.Tree(s.light_pos, s.intensity, topology="cost", cost_depth=depth)
    _check_tree(t)
    assert t.height <= depth + 96
    stack, checked = [(0, 1)], 0
    while stack:
        k, d = stack.pop()
        f, l, sp = int(t.first[k]), int(t.last[k]), int(t.split[k])
        if d <= depth:
            if d <= 2:
                assert sp == _rule(t.pos, t.inten, f, l)
        else:
            assert sp == _radix_rule(t.key, f, l)
            checked += 1
        for cf, cl, cid in ((f, sp, sp), (sp + 1, l, sp + 1)):
            if cf != cl:
                stack.append((cid, d + 1))
    assert checked > 0
