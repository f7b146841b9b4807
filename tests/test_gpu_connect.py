"""Connection evaluation through the C ABI against the oracle: per-pair weights and
visibility bits are bit-exact (the same float32 operations in the same order), per-eye
sums agree within the rounding of float32 accumulation."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, run_cull, upload_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    yield c
    c.close()


def _culled(ctx, s):
    g = upload_scene(s)
    ctx.set_shift_tile(s["tile"])
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
    st, cnt, pairs, _ = run_cull(ctx, g, tree, float(s["tau"]))
    tree.free()
    assert st == 0
    return g, pairs


def _connect(ctx, g, s, pairs, scene):
    import torch
    n = len(pairs)
    dp = torch.from_numpy(np.ascontiguousarray(pairs).view(np.int32)).to(dev())
    w = torch.zeros(max(n, 1), dtype=torch.float32, device=dev())
    v = torch.zeros(max(n, 1), dtype=torch.uint8, device=dev())
    sums = torch.zeros(len(s["eye_pos"]), dtype=torch.float32, device=dev())
    ctx.connect(g["ex"], g["ey"], g["ez"], (g["lx"], g["ly"], g["lz"], g["li"]), float(s["tau"]), dp, n,
                scene=scene, weight=w, visible=v, eye_sum=sums)
    return w[:n].cpu().numpy(), v[:n].cpu().numpy().astype(bool), sums.cpu().numpy()


def _check(s, pairs, got, tris):
    want = oracle.connect(s["eye_pos"], s["light_pos"], s["intensity"], pairs, s["tau"], tris)
    w, v, sums = got
    assert np.array_equal(v, want["visible"])
    assert np.array_equal(w.view(np.uint32), want["weight"].view(np.uint32))
    # float32 accumulation of n terms in any order: |error| <= (n + 1) 2^-23 |sum| (terms >= 0)
    per_eye = np.bincount(pairs[:, 0].astype(np.int64), minlength=len(sums))
    tol = (per_eye + 1) * 2.0 ** -23 * np.abs(want["eye_sum"]) + 1e-30
    assert np.all(np.abs(sums - want["eye_sum"]) <= tol)
    return want


@pytest.mark.parametrize("n_tris", [0, 1, 7, 5000])
def test_weights_and_visibility_equal_oracle(ctx, n_tris):
    import torch
    s = dict(synth.scene_frame(width=40, height=25, n_lights=6007, tile_w=16, tile_h=16, target=24.0, seed=81))
    g, pairs = _culled(ctx, s)
    tris = synth.occluder_triangles(n_tris, 82, size=0.02) if n_tris else None
    scene = ctx.build_scene(torch.from_numpy(tris).to(dev())) if n_tris else None
    want = _check(s, pairs, _connect(ctx, g, s, pairs, scene), tris)
    if n_tris == 5000:
        assert 0.1 < want["visible"].mean() < 0.9
    if scene is not None:
        scene.free()


def test_axis_aligned_segments_and_walls(ctx):
    # eyes and lights in the plane z = 0.5 (D.z = 0), walls of triangles along x and y
    import torch
    s = dict(synth.scene_uniform(n_lights=800, grid_w=16, grid_h=8, tile_w=8, tile_h=8, target=20.0, seed=83))
    s["eye_pos"] = s["eye_pos"].copy()
    s["light_pos"] = s["light_pos"].copy()
    s["eye_pos"][:, 2] = 0.5
    s["light_pos"][:, 2] = 0.5
    s["light_pos"][:40, 0] = s["eye_pos"][:40, 0]  # some segments also have D.x = 0
    g, pairs = _culled(ctx, s)
    walls = []
    for x0 in (0.25, 0.5, 0.75):  # vertical quads x = x0, two triangles each, half height
        walls += [[x0, 0.0, 0.25, x0, 0.6, 0.25, x0, 0.0, 0.75], [x0, 0.6, 0.25, x0, 0.6, 0.75, x0, 0.0, 0.75]]
    walls += [[0.0, 0.5, 0.5, 1.0, 0.5, 0.5, 0.0, 0.5, 0.9]]  # a wall y = 0.5 above the segments' plane
    walls += [[0.0, 0.0, 0.5, 1.0, 0.0, 0.5, 0.0, 1.0, 0.5]]  # in the segments' plane: det = 0, no hit
    tris = np.array(walls, np.float32)
    scene = ctx.build_scene(torch.from_numpy(tris).to(dev()))
    want = _check(s, pairs, _connect(ctx, g, s, pairs, scene), tris)
    assert 0.05 < want["visible"].mean() < 0.95
    scene.free()


def test_bad_inputs(ctx):
    import torch

    import paper_1907_12343_gb300 as hrr
    s = dict(synth.scene_uniform(n_lights=300, grid_w=8, grid_h=4, tile_w=8, tile_h=4, seed=84))
    g, pairs = _culled(ctx, s)
    bad = pairs.copy()
    bad[3, 1] = 300  # light id out of range
    with pytest.raises(hrr.HRRError) as e:
        _connect(ctx, g, s, bad, None)
    assert e.value.status == hrr.HRR_ERR_INVALID_ARG
    tris = synth.occluder_triangles(10, 85)
    tris[4, 2] = np.nan
    with pytest.raises(hrr.HRRError) as e:
        ctx.build_scene(torch.from_numpy(tris).to(dev()))
    assert e.value.status == hrr.HRR_ERR_INVALID_ARG
