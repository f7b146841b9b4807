"""Checks of the seeded input generators (CPU only)."""
import numpy as np

import synth


def test_splitmix64_published_vector():
    # splitmix64 seeded with 0 first adds the golden gamma and mixes it; the published
    # reference implementation's first output is 0xE220A8397B1DCDAF
    z = np.array([0x9E3779B97F4A7C15], dtype=np.uint64)
    assert int(synth._mix(z)[0]) == 0xE220A8397B1DCDAF


def test_streams_are_deterministic_and_distinct():
    a = synth.splitmix64(1, 0, 1000)
    assert np.array_equal(a, synth.splitmix64(1, 0, 1000))
    assert not np.array_equal(a, synth.splitmix64(1, 1, 1000))
    assert np.array_equal(a[500:], synth.splitmix64(1, 0, 500, offset=500))
    u = synth.uniform01(3, 4, 100000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_void_and_cluster_is_a_rank_permutation_with_blue_spectrum():
    r = synth.void_and_cluster(32, 32, 1)
    assert sorted(r.ravel().tolist()) == list(range(1024))
    # blue noise: thresholding at half the ranks leaves little low-frequency energy
    # compared with a white-noise permutation
    def low_energy(ranks):
        m = (ranks < ranks.size // 2).astype(float) - 0.5
        f = np.abs(np.fft.fft2(m)) ** 2
        fy = np.fft.fftfreq(ranks.shape[0])[:, None]
        fx = np.fft.fftfreq(ranks.shape[1])[None, :]
        low = (np.hypot(fx, fy) < 0.15) & (np.hypot(fx, fy) > 0)
        return f[low].mean()
    white = np.argsort(np.argsort(synth.uniform01(1, 99, 1024))).reshape(32, 32)
    assert low_energy(r) < 0.2 * low_energy(white)


def test_shift_tile_keeps_rank_order():
    t = synth.shift_tile(64, 64, 2).astype(np.uint64)
    ranks = synth.void_and_cluster(64, 64, 2)
    assert np.array_equal(t >> np.uint64(20), ranks.astype(np.uint64))
    assert len(np.unique(t)) == 4096


def test_rangemin_queries_shape():
    a, b, r = synth.rangemin_queries(200000, seed=3)
    a64, b64 = a.astype(np.int64), b.astype(np.int64)
    assert (b64 > a64).all() and (b64 <= 2**32 - 1).all()
    ln = b64 - a64
    # log-uniform lengths: roughly half the queries are at most 2^16 long
    assert 0.4 < (ln <= 65536).mean() < 0.65


def test_scene_shapes():
    s = synth.scene_uniform()
    assert s.light_pos.shape == (4096, 3) and s.eye_pos.shape == (1024, 3)
    assert s.light_pos.dtype == np.float32 and s.tile.dtype == np.uint32
    assert s.px.max() == 31 and s.py.max() == 31
    assert (s.light_pos >= 0).all() and (s.light_pos < 1).all()
    f = synth.scene_frame(width=40, height=30, n_lights=2000, tile_w=16, tile_h=16, seed=9)
    assert f.eye_pos.shape == (1200, 3) and f.light_pos.shape == (2000, 3)
    assert (f.light_pos >= 0).all() and (f.light_pos < 1).all()
    assert f.tau > 0
