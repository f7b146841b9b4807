"""GPU parity of several samples per light in one traversal (hrr_cull_samples, Sec. 3):
every sample's pairs equal the single-sample culling with that sample's shift (itself
pinned to the oracle), and the oracle's on the same shifts; the node visits summed over
the samples equal the single-sample totals."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, sorted_pairs, upload_scene

pytestmark = pytest.mark.gpu

PHI = 0x9E3779B9  # 2^32 / golden ratio: psi(n) = n PHI mod 2^32


@pytest.fixture(scope="module")
def ctx():
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    yield c
    c.close()


def _eyes(g, n=None):
    n = g["ex"].numel() if n is None else n
    return g["ex"][:n], g["ey"][:n], g["ez"][:n], g["px"][:n], g["py"][:n]


def _separate(ctx, g, tree, tau, offsets, cap, sample_indices=None):
    import torch
    out, visits = [], 0
    pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev())
    for s, off in enumerate(offsets):
        si = s if sample_indices is None else sample_indices[s]
        # binary records: the one-traversal samples kernel counts binary node visits
        st, cnt = ctx.cull(*_eyes(g), tree, tau, pairs, shift_offset=int(off) & 0xFFFFFFFF, sample_index=si,
                           tuning={"node_width": 2})
        assert st == 0
        out.append(sorted_pairs(pairs[:cnt].cpu().numpy().view(np.uint32)))
        visits += ctx.last_cull_stats()[0]
    return out, visits


def _fused(ctx, g, tree, tau, offsets, cap):
    import torch
    pairs = torch.empty((len(offsets), cap, 2), dtype=torch.int32, device=dev())
    st, counts, vis = ctx.cull_samples(*_eyes(g), tree, tau, offsets, pairs)
    got = [sorted_pairs(pairs[s, :min(c, cap)].cpu().numpy().view(np.uint32)) for s, c in enumerate(counts)]
    return st, counts, vis, got


@pytest.mark.parametrize("topology", ["radix", "cost"])
def test_psi_offsets_equal_separate_culls_and_oracle(ctx, topology):
    s = synth.scene_frame(width=257, height=131, n_lights=50021, tile_w=64, tile_h=64, target=64.0, seed=7)
    g = upload_scene(s)
    ctx.set_shift_tile(s.tile)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology=topology)
    offsets = [(n * PHI) & 0xFFFFFFFF for n in range(4)]
    cap = 256 * len(s.eye_pos)
    st, counts, (svis, fetched), got = _fused(ctx, g, tree, float(s.tau), offsets, cap)
    assert st == 0
    want, visits = _separate(ctx, g, tree, float(s.tau), offsets, cap)
    for s_, (a, b) in enumerate(zip(got, want)):
        assert counts[s_] == len(b) and np.array_equal(a, b), s_
    assert svis == visits
    assert fetched <= svis and fetched >= max(1, svis // len(offsets))
    # the oracle on sample 2: the tile rotated by psi(2)
    t = oracle.Tree(s.light_pos, s.intensity, topology=topology)
    rot = ((s.tile.astype(np.uint64) + offsets[2]) % (1 << 32)).astype(np.uint32)
    hier = oracle.cull_hier(t, s.eye_pos, s.px, s.py, rot, s.tau)
    assert np.array_equal(got[2], sorted_pairs(hier["pairs"]))
    tree.free()


def test_spacetime_layers_and_wraparound(ctx):
    # a 3-layer tile and 5 samples: sample s uses layer s mod 3 (and its own offset)
    s = synth.scene_frame(width=96, height=64, n_lights=20011, tile_w=32, tile_h=32, target=32.0, seed=12)
    g = upload_scene(s)
    t3 = synth.shift_tile_3d(32, 32, 4, 5)[:3].copy()
    ctx.set_shift_tile(t3)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology="cost")
    offsets = [0, 0, 0, 0, 12345]
    cap = 128 * len(s.eye_pos)
    st, counts, (svis, _), got = _fused(ctx, g, tree, float(s.tau), offsets, cap)
    assert st == 0
    want, visits = _separate(ctx, g, tree, float(s.tau), offsets, cap, sample_indices=[0, 1, 2, 3, 4])
    assert all(np.array_equal(a, b) for a, b in zip(got, want)) and svis == visits
    assert np.array_equal(got[0], got[3])  # layer 0 twice
    t = oracle.Tree(s.light_pos, s.intensity, topology="cost")
    hier = oracle.cull_hier(t, s.eye_pos, s.px, s.py, t3, s.tau, sample_index=1)
    assert np.array_equal(got[1], sorted_pairs(hier["pairs"]))
    ctx.set_shift_tile(s.tile)
    tree.free()


@pytest.mark.parametrize("n_samples", [1, 32])
def test_one_and_thirty_two_samples(ctx, n_samples):
    s = synth.scene_uniform(n_lights=4096, seed=31)
    g = upload_scene(s)
    ctx.set_shift_tile(s.tile)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    offsets = [(n * PHI) & 0xFFFFFFFF for n in range(n_samples)]
    cap = 64 * len(s.eye_pos)
    st, counts, (svis, fetched), got = _fused(ctx, g, tree, float(s.tau), offsets, cap)
    assert st == 0
    want, visits = _separate(ctx, g, tree, float(s.tau), offsets, cap)
    assert all(np.array_equal(a, b) for a, b in zip(got, want)) and svis == visits
    if n_samples == 1:
        assert fetched == svis
        t = oracle.Tree(s.light_pos, s.intensity)
        flat = oracle.cull_flat(t, s.eye_pos, s.px, s.py, s.tile, s.tau)
        assert np.array_equal(got[0], sorted_pairs(flat["pairs"]))
    tree.free()


def test_overflow_zero_eyes_and_bad_args(ctx):
    import torch
    import paper_1907_12343_gb300 as hrr
    s = synth.scene_frame(width=120, height=80, n_lights=5003, tile_w=16, tile_h=16, target=24.0, seed=9)
    g = upload_scene(s)
    ctx.set_shift_tile(s.tile)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology="cost")
    offsets = [0, PHI, (2 * PHI) & 0xFFFFFFFF]
    st, need, _, full = _fused(ctx, g, tree, float(s.tau), offsets, 64 * len(s.eye_pos))
    assert st == 0
    small = min(need) // 2
    st, counts, _, part = _fused(ctx, g, tree, float(s.tau), offsets, small)
    assert st == hrr.HRR_ERR_OVERFLOW and counts == need
    for a, b in zip(part, full):  # the pairs that fit are accepted pairs of their sample
        key = lambda p: (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)
        kb = np.sort(key(b))
        ka = key(a)
        assert len(ka) == small and np.array_equal(kb[np.minimum(np.searchsorted(kb, ka), len(kb) - 1)], ka)
    pairs = torch.empty((3, 16, 2), dtype=torch.int32, device=dev())
    st, counts, vis = ctx.cull_samples(*_eyes(g, 0), tree, float(s.tau), offsets, pairs)
    assert st == 0 and counts == [0, 0, 0] and vis == (0, 0)
    for bad in ([], list(range(33))):
        with pytest.raises(hrr.HRRError):
            ctx.cull_samples(*_eyes(g), tree, float(s.tau), bad, torch.empty((max(len(bad), 1), 16, 2),
                                                                                 dtype=torch.int32, device=dev()))
    tree.free()


def test_full_frame_four_samples(ctx):
    # the benchmark's frame (1920 x 1080 eyes, 2^20 cost-driven lights) with four psi(n)
    # samples: every sample's whole set equals its single-sample culling
    import torch
    s = synth.scene_frame()
    g = upload_scene(s)
    ctx.set_shift_tile(s.tile)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology="cost")
    offsets = [(n * PHI) & 0xFFFFFFFF for n in range(4)]
    n_e = len(s.eye_pos)
    cap = 80 * n_e
    pairs = torch.empty((4, cap, 2), dtype=torch.int32, device=dev())
    st, counts, (svis, fetched) = ctx.cull_samples(*_eyes(g), tree, float(s.tau), offsets, pairs)
    assert st == 0

    def keys(p):
        p = p.to(torch.int64)
        return torch.sort((p[:, 0] << 32) | (p[:, 1] & 0xFFFFFFFF)).values

    single = torch.empty((cap, 2), dtype=torch.int32, device=dev())
    total = 0
    for k, off in enumerate(offsets):
        st1, cnt = ctx.cull(*_eyes(g), tree, float(s.tau), single, shift_offset=off, tuning={"node_width": 2})
        assert st1 == 0 and cnt == counts[k]
        assert torch.equal(keys(pairs[k, :cnt]), keys(single[:cnt]))
        total += ctx.last_cull_stats()[0]
    assert svis == total and fetched < svis
    tree.free()
