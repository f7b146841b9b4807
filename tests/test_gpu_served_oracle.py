"""Served culling checked against the oracle itself, not against plain hrr_cull.

Jobs of different sizes, trees and shift sources arrive while others run (small slices
force them to share traversal launches), and every job's pairs equal the oracle's:
the flat brute force for the small jobs (whole, or eye sub-ranges with a shift offset),
a job that refits its own hierarchy to moved lights (against the oracle's refit), a job
on a space-time tile at a sample index, and a frame-sized job (1920 x 1080 eyes x 2^20
lights over the cost-driven hierarchy) on sampled eyes against the hierarchical oracle
and, for a few of them, the flat brute force.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, oracle_hier, sorted_pairs, upload_scene

pytestmark = pytest.mark.gpu


def _tile_dev(tile):
    import torch
    return torch.from_numpy(np.ascontiguousarray(tile, dtype=np.uint32).view(np.int32)).to(dev())


def _moved(pos, inten, seed, scale=0.04):
    jitter = (synth.uniform01(seed, 1, 3 * len(pos)).reshape(-1, 3) - 0.5) * scale
    p = np.clip(pos + jitter.astype(np.float32), 0.0, 1.0).astype(np.float32)
    i = (inten * (0.5 + synth.uniform01(seed, 2, len(inten)))).astype(np.float32)
    return p, i


def _job_pairs(srv, t, r):
    import paper_1907_12343_gb300 as hrr
    assert r["wait_status"] == hrr.HRR_OK and r["status"] == hrr.HRR_OK, r
    got = srv.pairs(t, r)
    assert len(got) == r["count"]
    return sorted_pairs(got)


def test_served_jobs_equal_the_oracle():
    import torch

    import paper_1907_12343_gb300 as hrr
    ctx = hrr.Context(0)
    small = [dict(synth.scene_uniform()),
             dict(synth.scene_frame(width=61, height=37, n_lights=5003, tile_w=16, tile_h=16, target=48.0, seed=5)),
             dict(synth.scene_frame(width=257, height=131, n_lights=50021, tile_w=64, tile_h=64, target=64.0,
                                    seed=7))]
    gs = [upload_scene(s) for s in small]
    trees = [ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology=topo)
             for g, topo in zip(gs, ("radix", "cost", "cost"))]
    tiles = [_tile_dev(s["tile"]) for s in small]
    # the refitting job's own hierarchy (built on scene 1's lights, refit to moved lights)
    s_r = small[1]
    g_r = gs[1]
    tree_r = ctx.build_light_tree(g_r["lx"], g_r["ly"], g_r["lz"], g_r["li"], topology="cost")
    mpos, minten = _moved(s_r["light_pos"], s_r["intensity"], seed=61)
    mp = torch.from_numpy(mpos).to(dev())
    moved = [mp[:, 0].contiguous(), mp[:, 1].contiguous(), mp[:, 2].contiguous(),
             torch.from_numpy(minten).to(dev())]
    # a space-time tile for scene 2's eyes
    t3 = synth.shift_tile_3d(16, 16, 4, seed=62)
    t3_dev = _tile_dev(t3)
    # the frame-sized job
    big = synth.scene_frame()
    g_big = upload_scene(big)
    tree_big = ctx.build_light_tree(g_big["lx"], g_big["ly"], g_big["lz"], g_big["li"], topology="cost")

    srv = hrr.Server(ctx, hbm_budget_bytes=16 << 30, slice_eyes=1 << 16)
    jobs = []  # (ticket, kind, details)

    def submit(g, tree, tau, a, b, tile, cap=None, **kw):
        return srv.submit(g["ex"][a:b], g["ey"][a:b], g["ez"][a:b], g["px"][a:b], g["py"][a:b], tree, float(tau),
                          cap or 256 * (b - a) + 1024, tile=tile, **kw)

    n_big = len(big.eye_pos)
    jobs.append((submit(g_big, tree_big, big.tau, 0, n_big, _tile_dev(big.tile), cap=200 * n_big), "big", None))
    for k, (si, a, b, off) in enumerate([(0, 0, 1024, 0), (1, 0, 2257, 0x9E3779B9), (2, 1000, 30000, 0),
                                         (0, 100, 900, 12345), (2, 0, 33667, 0), (1, 500, 1500, 0)]):
        n_e = len(small[si]["eye_pos"])
        b = min(b, n_e)
        jobs.append((submit(gs[si], trees[si], small[si]["tau"], a, b, tiles[si], shift_offset=off),
                     "small", (si, a, b, off)))
        if k % 2 == 1:
            time.sleep(0.003)  # later jobs arrive while earlier ones are on the GPU
    jobs.append((submit(g_r, tree_r, s_r["tau"], 0, len(s_r["eye_pos"]), tiles[1], refit=moved), "refit", None))
    jobs.append((submit(gs[2], trees[2], small[2]["tau"], 0, 20000, t3_dev, sample_index=5), "spacetime", None))

    for t, kind, info in jobs:
        r = srv.wait(t, 600.0)
        got = _job_pairs(srv, t, r)
        if kind == "small":
            si, a, b, off = info
            s = small[si]
            to = oracle.Tree(s["light_pos"], s["intensity"], topology=("radix", "cost", "cost")[si])
            tile = (np.asarray(s["tile"], np.uint64) + off).astype(np.uint32)
            ids = np.arange(a, b, dtype=np.uint32)
            flat = oracle.cull_flat(to, s["eye_pos"][a:b], s["px"][a:b], s["py"][a:b], tile, s["tau"])
            assert np.array_equal(got, sorted_pairs(flat["pairs"])), info
            assert len(ids) == b - a
        elif kind == "refit":
            to = oracle.Tree(s_r["light_pos"], s_r["intensity"], topology="cost")
            to.refit(mpos, minten)
            flat = oracle.cull_flat(to, s_r["eye_pos"], s_r["px"], s_r["py"], s_r["tile"], s_r["tau"])
            assert np.array_equal(got, sorted_pairs(flat["pairs"]))
        elif kind == "spacetime":
            s = small[2]
            to = oracle.Tree(s["light_pos"], s["intensity"], topology="cost")
            flat = oracle.cull_flat(to, s["eye_pos"][:20000], s["px"][:20000], s["py"][:20000], t3, s["tau"],
                                    sample_index=5)
            assert np.array_equal(got, sorted_pairs(flat["pairs"]))
        else:
            ids = np.unique(np.concatenate([np.arange(0, n_big, n_big // 151), [n_big - 1]])).astype(np.uint32)
            to = oracle.Tree(big.light_pos, big.intensity, topology="cost")
            hier = oracle_hier(to, big.eye_pos[ids], big.px[ids], big.py[ids], big.tile, big.tau, eye_ids=ids)
            sel = got[np.isin(got[:, 0], ids)]
            assert np.array_equal(sel, sorted_pairs(hier["pairs"]))
            few = ids[::15]
            flat = oracle.cull_flat(to, big.eye_pos[few], big.px[few], big.py[few], big.tile, big.tau, eye_ids=few)
            assert np.array_equal(got[np.isin(got[:, 0], few)], sorted_pairs(flat["pairs"]))
            assert 20 * n_big < len(got) < 200 * n_big
        srv.release(t)
    st = srv.stats()
    assert st["jobs_done"] == len(jobs) and st["max_active"] > 1
    srv.destroy()
    for tr in trees + [tree_r, tree_big]:
        tr.free()
    ctx.close()
