"""GPU parity of the light hierarchy: Morton order, radix-tree topology, boxes and maximum
intensities equal the oracle's top-down build, node by node (bit-exact)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import upload_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    yield c
    c.close()


def _compare(ctx, pos, inten):
    g = upload_scene({"light_pos": pos, "intensity": inten, "eye_pos": pos[:1], "px": np.zeros(1, np.uint16),
                      "py": np.zeros(1, np.uint16)})
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    nodes, perm = tree.download()
    t = oracle.Tree(pos, inten)
    assert np.array_equal(perm, t.perm)
    assert tree.height == t.height
    n = len(inten)
    if n == 1:
        tree.free()
        return
    first = np.minimum(np.arange(n - 1), nodes["other_end"])
    last = np.maximum(np.arange(n - 1), nodes["other_end"])
    assert np.array_equal(first, t.first) and np.array_equal(last, t.last)
    assert np.array_equal(nodes["split"], t.split)
    s = nodes["split"].astype(np.int64)
    for c, cid, leaf in ((0, s, first == s), (1, s + 1, last == s + 1)):
        lo = nodes[f"c{c}_lo"]
        hi = nodes[f"c{c}_hi"]
        im = nodes[f"c{c}_imax"]
        li = cid[leaf]
        assert np.array_equal(lo[leaf], t.pos[li]) and np.array_equal(hi[leaf], t.pos[li])
        assert np.array_equal(im[leaf], t.inten[li])
        ii = cid[~leaf]
        assert np.array_equal(lo[~leaf], t.lo[ii]) and np.array_equal(hi[~leaf], t.hi[ii])
        assert np.array_equal(im[~leaf], t.imax[ii])
    tree.free()


@pytest.mark.parametrize("n", [1, 2, 3, 5, 64, 1000, 4097])
def test_uniform_lights(ctx, n):
    rng = np.random.default_rng(n)
    pos = rng.random((n, 3)).astype(np.float32)
    inten = np.exp(rng.standard_normal(n)).astype(np.float32)
    _compare(ctx, pos, inten)


def test_duplicate_keys(ctx):
    rng = np.random.default_rng(3)
    pos = (rng.integers(0, 4, (20000, 3)) / 4.0).astype(np.float32)
    _compare(ctx, pos, rng.random(20000).astype(np.float32))
    _compare(ctx, np.full((777, 3), 0.3, np.float32), np.ones(777, np.float32))


def test_outside_unit_cube_is_clamped(ctx):
    rng = np.random.default_rng(4)
    pos = (rng.random((5000, 3)) * 3 - 1).astype(np.float32)
    _compare(ctx, pos, rng.random(5000).astype(np.float32))


def test_gaussian_mixture_ragged(ctx):
    pos = synth.gaussian_mixture_lights(100003, 64, seed=5)
    inten = np.exp(1.5 * synth.normal(5, 6, 100003)).astype(np.float32)
    _compare(ctx, pos, inten)


def test_full_size_frame_lights(ctx):
    s = synth.scene_frame()
    _compare(ctx, s.light_pos, s.intensity)


@pytest.mark.parametrize("topology", ["radix", "cost"])
def test_nonfinite_lights_rejected(ctx, topology):
    # for the cost-driven build, 5,000 lights reach every split kernel; an infinite
    # intensity makes the cost of every split of a range holding it NaN (such ranges then
    # split at their first light down to the cost depth), and the build still ends and
    # reports the input
    import paper_1907_12343_gb300 as hrr
    n = 5000 if topology == "cost" else 100
    pos = np.random.default_rng(1).random((n, 3)).astype(np.float32)
    inten = np.ones(n, np.float32)
    for bad in ("pos", "inten", "all_nan"):
        p, i = pos.copy(), inten.copy()
        if bad == "pos":
            p[17, 1] = np.nan
        elif bad == "inten":
            i[42] = np.inf
        else:
            i[:] = np.nan
        g = upload_scene({"light_pos": p, "intensity": i, "eye_pos": p[:1], "px": np.zeros(1, np.uint16),
                          "py": np.zeros(1, np.uint16)})
        with pytest.raises(hrr.HRRError) as e:
            ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology=topology)
        assert e.value.status == hrr.HRR_ERR_INVALID_ARG


@pytest.mark.parametrize("topology", ["radix", "cost"])
def test_build_from_host_lights_equals_device_build(ctx, topology):
    # hrr_build_light_tree_host stages host lights itself; the hierarchy is the same
    import torch
    s = synth.scene_frame(width=8, height=8, n_lights=70001, tile_w=8, tile_h=8, seed=81)
    g = upload_scene(s)
    ref = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology=topology)
    host = [torch.from_numpy(np.ascontiguousarray(s.light_pos[:, k])).pin_memory() for k in range(3)]
    host.append(torch.from_numpy(np.ascontiguousarray(s.intensity)).pin_memory())
    for _ in range(2):  # the staging area is reused
        t = ctx.build_light_tree_host(*host, topology=topology)
        a, pa = t.download()
        b, pb = ref.download()
        assert a.tobytes() == b.tobytes() and np.array_equal(pa, pb) and t.height == ref.height
        t.free()
    # pageable numpy arrays work too
    t = ctx.build_light_tree_host(*[np.ascontiguousarray(s.light_pos[:, k]) for k in range(3)],
                                  np.ascontiguousarray(s.intensity), topology=topology)
    assert t.download()[0].tobytes() == ref.download()[0].tobytes()
    t.free()
    ref.free()
