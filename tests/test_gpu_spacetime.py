"""Space-time shifts psi(j, n) from a 3D tile (Sec. 3) through the C ABI: sample n of every
eye uses layer n mod d, for the plain call, batches and the server, against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, oracle_hier, run_cull, sorted_pairs, upload_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import paper_1907_12343_gb300 as hrr
    ctx = hrr.Context(0)
    s = synth.scene_frame(width=57, height=23, n_lights=9001, tile_w=16, tile_h=16, target=24.0, seed=51)
    t3 = synth.shift_tile_3d(16, 16, 4, seed=52)
    g = upload_scene(s)
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    yield hrr, ctx, s, t3, g, tree
    tree.free()
    ctx.close()


def _plain(ctx, g, tree, tau, n, **kw):
    import torch
    cap = 256 * g["ex"].numel()
    pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev())
    vis = torch.zeros(g["ex"].numel(), dtype=torch.int32, device=dev())
    st, cnt = ctx.cull(g["ex"], g["ey"], g["ez"], g["px"], g["py"], tree, tau, pairs, eye_visits=vis,
                       sample_index=n, **kw)
    assert st == 0
    return sorted_pairs(pairs[:cnt].cpu().numpy().view(np.uint32)), vis.cpu().numpy().view(np.uint32)


def test_samples_use_their_layer(env):
    hrr, ctx, s, t3, g, tree = env
    ctx.set_shift_tile(t3)
    t = oracle.Tree(s.light_pos, s.intensity)
    for n in (0, 1, 3, 6):
        pairs, vis = _plain(ctx, g, tree, float(s.tau), n)
        flat = oracle.cull_flat(t, s.eye_pos, s.px, s.py, t3, s.tau, sample_index=n)
        hier = oracle_hier(t, s.eye_pos, s.px, s.py, t3, s.tau, sample_index=n)
        assert np.array_equal(pairs, sorted_pairs(flat["pairs"]))
        assert np.array_equal(vis, hier["visits"].astype(np.uint32))


def test_lattice_tile_equals_shift_offset(env):
    # layers tile + n / phi (mod 1): sample n equals the plain tile with psi(n) = n / phi
    hrr, ctx, s, t3, g, tree = env
    alpha = 0x9E3779B9
    lat = np.stack([(s.tile.astype(np.uint64) + n * alpha) % (1 << 32) for n in range(5)]).astype(np.uint32)
    for n in (2, 4):
        ctx.set_shift_tile(lat)
        a, va = _plain(ctx, g, tree, float(s.tau), n)
        ctx.set_shift_tile(s.tile)
        b, vb = _plain(ctx, g, tree, float(s.tau), 0, shift_offset=(n * alpha) & 0xFFFFFFFF)
        assert np.array_equal(a, b) and np.array_equal(va, vb)


def test_batch_and_server_frames_pick_their_layers(env):
    import torch
    hrr, ctx, s, t3, g, tree = env
    dev_t3 = torch.from_numpy(t3.view(np.int32)).to(dev())
    ctx.set_shift_tile(t3)
    want = {n: _plain(ctx, g, tree, float(s.tau), n)[0] for n in range(4)}
    frames = []
    for k, n in enumerate((0, 3, 5, 2)):
        cnt = len(want[n % 4])
        frames.append({"x": g["ex"], "y": g["ey"], "z": g["ez"], "px": g["px"], "py": g["py"], "tree": tree,
                       "tau": float(s.tau), "sample_index": n, "tile": dev_t3 if k % 2 else None,
                       "pairs": torch.empty((cnt + 16, 2), dtype=torch.int32, device=dev())})
    b = hrr.Batch(ctx, frames, use_graph=True)
    b.launch()
    st, counts, _ = b.results()
    assert st == hrr.HRR_OK
    for fr, c in zip(frames, counts):
        got = sorted_pairs(fr["pairs"][:c].cpu().numpy().view(np.uint32))
        assert np.array_equal(got, want[fr["sample_index"] % 4])
    b.destroy()
    srv = hrr.Server(ctx, hbm_budget_bytes=1 << 30)
    tickets = []
    for k, n in enumerate((1, 6, 3)):
        tickets.append((n, srv.submit(g["ex"], g["ey"], g["ez"], g["px"], g["py"], tree, float(s.tau),
                                      len(want[n % 4]) + 16, tile=dev_t3 if k % 2 else None, sample_index=n)))
    for n, t in tickets:
        r = srv.wait(t, 120.0)
        assert r["status"] == hrr.HRR_OK
        assert np.array_equal(sorted_pairs(srv.pairs(t, r)), want[n % 4])
        srv.release(t)
    srv.destroy()
