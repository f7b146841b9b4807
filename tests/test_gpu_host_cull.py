"""GPU parity of culling with host buffers (hrr_cull_host): eyes read from host memory,
pairs written to host memory, the eyes culled in slices whose copies overlap the culling.
The accepted set must equal the oracle's (Sec. 1) exactly, as for hrr_cull."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import oracle_hier, sorted_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    yield c
    c.close()


def _host_eyes(s, pinned):
    import torch
    ep = np.ascontiguousarray(s["eye_pos"], dtype=np.float32)
    arrs = [np.ascontiguousarray(ep[:, k]) for k in range(3)]
    arrs += [np.ascontiguousarray(s["px"]).view(np.int16), np.ascontiguousarray(s["py"]).view(np.int16)]
    if not pinned:
        return arrs
    return [torch.from_numpy(a).pin_memory() for a in arrs]


def _tree(ctx, s, topology="radix"):
    import torch
    d = torch.device("cuda:0")
    lp = torch.from_numpy(np.ascontiguousarray(s["light_pos"])).to(d)
    L = [lp[:, k].contiguous() for k in range(3)] + [torch.from_numpy(np.ascontiguousarray(s["intensity"])).to(d)]
    return ctx.build_light_tree(*L, topology=topology), L


def _host_pairs(cap, pinned):
    import torch
    p = torch.empty((cap, 2), dtype=torch.int32)
    return p.pin_memory() if pinned else p


@pytest.mark.parametrize("pinned", [True, False])
def test_ragged_frame_equals_oracle(ctx, pinned):
    s = dict(synth.scene_frame(width=257, height=131, n_lights=50021, tile_w=64, tile_h=64, target=64.0, seed=7))
    ctx.set_shift_tile(s["tile"])
    tree, _ = _tree(ctx, s)
    pairs = _host_pairs(256 * len(s["eye_pos"]), pinned)
    st, cnt = ctx.cull_host(*_host_eyes(s, pinned), tree, float(s["tau"]), pairs)
    tree.free()
    assert st == 0
    t = oracle.Tree(s["light_pos"], s["intensity"])
    hier = oracle_hier(t, s["eye_pos"], s["px"], s["py"], s["tile"], s["tau"])
    got = pairs[:cnt].numpy().view(np.uint32)
    assert np.array_equal(sorted_pairs(got), sorted_pairs(hier["pairs"]))


def test_eight_slices_equal_device_cull_and_oracle(ctx):
    # 1920 x 1080 eyes (eight slices on two streams) over 2^16 cost-driven lights: the whole
    # set equals the device-buffer cull's, sampled eyes equal the oracle's, and so do the
    # node visits
    import torch
    s = dict(synth.scene_frame(width=1920, height=1080, n_lights=1 << 16, tile_w=64, tile_h=64, target=24.0, seed=21))
    n_e = len(s["eye_pos"])
    ctx.set_shift_tile(s["tile"])
    tree, _ = _tree(ctx, s, topology="cost")
    cap = 40 * n_e
    hp = _host_pairs(cap, True)
    st, cnt = ctx.cull_host(*_host_eyes(s, True), tree, float(s["tau"]), hp)
    assert st == 0 and 0 < cnt <= cap
    visits_host, acc_host = ctx.last_cull_stats()
    assert acc_host == cnt
    d = torch.device("cuda:0")
    eh = _host_eyes(s, False)
    dev_e = [torch.from_numpy(a).to(d) for a in eh]
    dp = torch.empty((cap, 2), dtype=torch.int32, device=d)
    st2, cnt2 = ctx.cull(*dev_e, tree, float(s["tau"]), dp)
    assert st2 == 0 and cnt2 == cnt
    assert ctx.last_cull_stats()[0] == visits_host

    def keys(p):
        p = p.to(torch.int64)
        return torch.sort((p[:, 0] << 32) | (p[:, 1] & 0xFFFFFFFF)).values

    assert torch.equal(keys(hp[:cnt].to(d)), keys(dp[:cnt]))
    got = hp[:cnt].numpy().view(np.uint32)
    assert got[:, 0].max() < n_e and np.bincount(got[:, 0], minlength=n_e).sum() == cnt
    ids = np.unique(np.concatenate([np.arange(0, n_e, n_e // 97), [n_e - 1]])).astype(np.uint32)
    t = oracle.Tree(s["light_pos"], s["intensity"], topology="cost")
    hier = oracle_hier(t, s["eye_pos"][ids], s["px"][ids], s["py"][ids], s["tile"], s["tau"], eye_ids=ids)
    assert np.array_equal(sorted_pairs(got[np.isin(got[:, 0], ids)]), sorted_pairs(hier["pairs"]))
    tree.free()


def test_overflow_zero_eyes_and_bad_args(ctx):
    import paper_1907_12343_gb300 as hrr
    # 700 x 600 eyes: two slices, so the overflow spans both pair buffers
    s = dict(synth.scene_frame(width=700, height=600, n_lights=4001, tile_w=16, tile_h=16, target=32.0, seed=5))
    ctx.set_shift_tile(s["tile"])
    tree, _ = _tree(ctx, s)
    eyes = _host_eyes(s, True)
    full = _host_pairs(64 * len(s["eye_pos"]), True)
    st, need = ctx.cull_host(*eyes, tree, float(s["tau"]), full)
    assert st == 0
    small = _host_pairs(need // 3, True)
    st, cnt = ctx.cull_host(*eyes, tree, float(s["tau"]), small)
    assert st == hrr.HRR_ERR_OVERFLOW and cnt == need
    # the pairs that fit are distinct accepted pairs
    key = lambda p: (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)
    whole = np.sort(key(full[:need].numpy().view(np.uint32)))
    part = key(small.numpy().view(np.uint32))
    assert len(np.unique(part)) == len(part)
    pos = np.minimum(np.searchsorted(whole, part), len(whole) - 1)
    assert np.array_equal(whole[pos], part)
    empty = [a[:0] for a in eyes]
    st, cnt = ctx.cull_host(*empty, tree, float(s["tau"]), full)
    assert st == 0 and cnt == 0
    with pytest.raises(hrr.HRRError):
        ctx.cull_host(*eyes, tree, float("nan"), full)
    tree.free()
