"""Served culling (continuous batching) through the C ABI: every job's result is the same
when it runs in a mix of concurrently admitted jobs as when it runs alone (plain
hrr_cull), under budget-limited admission and with jobs arriving while others run."""
import time

import numpy as np
import pytest

import synth
from gpu_util import dev, run_cull, sorted_pairs, upload_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1907_12343_gb300 as hrr
    ctx = hrr.Context(0)
    scenes = [
        dict(synth.scene_frame(width=257, height=131, n_lights=50021, tile_w=64, tile_h=64,
                               target=64.0, seed=7)),
        dict(synth.scene_frame(width=200, height=100, n_lights=20000, tile_w=64, tile_h=64,
                               target=24.0, seed=8)),
        dict(synth.scene_uniform()),
    ]
    trees, gs, tiles = [], [], []
    for s in scenes:
        g = upload_scene(s)
        gs.append(g)
        trees.append(ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"]))
        tiles.append(torch.from_numpy(np.ascontiguousarray(s["tile"]).view(np.int32)).to(dev()))
    yield hrr, ctx, scenes, gs, trees, tiles
    for t in trees:
        t.free()
    ctx.close()


def _jobs(scenes, gs):
    rng = np.random.default_rng(5)
    jobs = []
    for k in range(12):
        si = k % 3
        n_e = len(scenes[si]["eye_pos"])
        a = int(rng.integers(0, n_e // 2))
        b = int(rng.integers(a + 1, n_e + 1))
        if k == 5:
            a, b = 0, n_e  # one whole frame
        off = int(rng.integers(0, 2**32)) if k % 4 == 1 else 0
        jobs.append((si, a, b, off))
    return jobs


def _alone(hrr, ctx, scenes, gs, trees, si, a, b, off):
    ctx.set_shift_tile(scenes[si]["tile"])
    g = {k: v[a:b] if k.startswith("e") or k in ("px", "py") else v for k, v in gs[si].items()}
    st, cnt, pairs, _ = run_cull(ctx, g, trees[si], float(scenes[si]["tau"]), shift_offset=off)
    assert st == hrr.HRR_OK
    return pairs


def _submit(srv, gs, trees, tiles, scenes, si, a, b, off, cap=None):
    g = gs[si]
    n = b - a
    return srv.submit(g["ex"][a:b], g["ey"][a:b], g["ez"][a:b], g["px"][a:b], g["py"][a:b], trees[si],
                      float(scenes[si]["tau"]), cap if cap is not None else 256 * n, tile=tiles[si],
                      shift_offset=off)


def test_jobs_in_the_mix_equal_alone(env):
    hrr, ctx, scenes, gs, trees, tiles = env
    srv = hrr.Server(ctx, hbm_budget_bytes=8 << 30, slice_eyes=1 << 15)
    jobs = _jobs(scenes, gs)
    tickets = []
    for k, job in enumerate(jobs):
        tickets.append(_submit(srv, gs, trees, tiles, scenes, *job))
        if k % 4 == 3:
            time.sleep(0.002)  # later jobs arrive while earlier ones are on the GPU
    for t, job in zip(tickets, jobs):
        r = srv.wait(t, 300.0)
        assert r["wait_status"] == hrr.HRR_OK and r["status"] == hrr.HRR_OK
        got = srv.pairs(t, r)
        assert len(got) == r["count"]
        ref = _alone(hrr, ctx, scenes, gs, trees, *job)
        assert np.array_equal(sorted_pairs(got), sorted_pairs(ref))
        srv.release(t)
    st = srv.stats()
    assert st["jobs_done"] == len(jobs) and st["max_active"] > 1 and st["slices"] > 1
    srv.destroy()


def test_budget_limits_concurrency(env):
    hrr, ctx, scenes, gs, trees, tiles = env
    jobs = [(0, 0, 20000, 0), (1, 0, 15000, 3), (2, 0, 1024, 0), (0, 5000, 30000, 9), (1, 100, 9000, 0)]
    cap = 20000 * 256
    srv = hrr.Server(ctx, hbm_budget_bytes=2 * cap * 8, slice_eyes=1 << 14)
    tickets = [_submit(srv, gs, trees, tiles, scenes, *j, cap=cap) for j in jobs]
    for t, job in zip(tickets, jobs):
        r = srv.wait(t, 300.0)
        assert r["status"] == hrr.HRR_OK
        ref = _alone(hrr, ctx, scenes, gs, trees, *job)
        assert np.array_equal(sorted_pairs(srv.pairs(t, r)), sorted_pairs(ref))
        srv.release(t)
    assert srv.stats()["max_active"] <= 2
    srv.destroy()


def test_refused_overflowing_and_empty_jobs(env):
    hrr, ctx, scenes, gs, trees, tiles = env
    srv = hrr.Server(ctx, hbm_budget_bytes=64 << 20)
    too_big = _submit(srv, gs, trees, tiles, scenes, 0, 0, 1000, 0, cap=(64 << 20) // 8 + 1)
    small = _submit(srv, gs, trees, tiles, scenes, 0, 0, 2000, 0, cap=100)
    empty = _submit(srv, gs, trees, tiles, scenes, 2, 0, 0, 0, cap=0)
    fine = _submit(srv, gs, trees, tiles, scenes, 2, 0, 1024, 0)
    assert srv.wait(too_big, 60.0)["status"] == hrr.HRR_ERR_OOM
    r = srv.wait(small, 60.0)
    assert r["status"] == hrr.HRR_ERR_OVERFLOW
    ref = _alone(hrr, ctx, scenes, gs, trees, 0, 0, 2000, 0)
    assert r["count"] == len(ref) and len(srv.pairs(small, r)) == 100
    r = srv.wait(empty, 60.0)
    assert r["status"] == hrr.HRR_OK and r["count"] == 0
    r = srv.wait(fine, 60.0)
    assert r["status"] == hrr.HRR_OK
    for t in (too_big, small, empty, fine):
        srv.release(t)
    srv.destroy()


def test_wait_times_out_then_completes(env):
    hrr, ctx, scenes, gs, trees, tiles = env
    srv = hrr.Server(ctx, hbm_budget_bytes=8 << 30)
    t = _submit(srv, gs, trees, tiles, scenes, 0, 0, len(scenes[0]["eye_pos"]), 0)
    first = srv.wait(t, 0.0)
    assert first["wait_status"] in (hrr.HRR_ERR_TIMEOUT, hrr.HRR_OK)
    if first["wait_status"] == hrr.HRR_ERR_TIMEOUT:
        assert first["status"] == hrr.HRR_PENDING
    r = srv.wait(t, 120.0)
    assert r["wait_status"] == hrr.HRR_OK and r["status"] == hrr.HRR_OK
    srv.release(t)
    with pytest.raises(hrr.HRRError):
        srv.release(t)  # unknown ticket now
    srv.destroy()
