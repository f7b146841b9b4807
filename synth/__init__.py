"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module draws random numbers and shapes workloads; it holds none of the culling
method's arithmetic (no radical inverse, no range minimum, no acceptance test). Every
array is a deterministic function of its seed, built from one counter-based generator:

* splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
  OOPSLA 2014): the output of counter k of stream s is mix(key(seed, s) + (k+1)*golden),
  with the published mixing function and golden gamma 0x9E3779B97F4A7C15.
* Uniform doubles take the top 53 bits; normals use the Box-Muller transform.

Workloads (shapes and distributions of the paper's setting: eye vertices sorted by pixel,
light vertices spread over a scene, one blue-noise Cranley-Patterson shift per pixel,
Sec. 1 of the paper):

* ``scene_uniform``: lights and eyes uniform in the unit cube, eyes on a pixel grid.
* ``scene_frame``: eyes of a WxH frame jittered onto a heightfield, lights from an
  isotropic Gaussian mixture clipped to the unit cube, lognormal intensities.
* ``rangemin_queries``: (a, b, r) triples with log-uniform range lengths.
* ``shift_tile``: void-and-cluster blue-noise ranks (Ulichney 1993) dithered to 32 bits.
* ``calibrate_tau``: picks the culling scale tau so that the expected number of
  accepted lights per eye, averaged over a fixed eye sample, hits a target.
"""
from __future__ import annotations

import functools
import math

import numpy as np

__all__ = [
    "splitmix64",
    "uniform01",
    "normal",
    "void_and_cluster",
    "shift_tile",
    "calibrate_tau",
    "scene_uniform",
    "scene_frame",
    "rangemin_queries",
    "Scene",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` uint64 outputs of stream ``stream`` under ``seed``, counters offset.. offset+n-1."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) * _GOLDEN
                   + np.uint64(stream & 0xFFFFFFFFFFFFFFFF))[0]
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(key + ctr * _GOLDEN)


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform float64 in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller; uses counters 2*offset .. 2*(offset+n)-1."""
    u = uniform01(seed, stream, 2 * n, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


_ONE_BELOW = np.float32(np.nextafter(np.float32(1.0), np.float32(0.0)))


def _to_unit_f32(x: np.ndarray) -> np.ndarray:
    """float64 in [0,1) -> float32 in [0,1) (rounding can reach 1.0f; clamp below it)."""
    return np.minimum(x.astype(np.float32), _ONE_BELOW)


# --------------------------------------------------------------------------------------
# Blue-noise shift tile
# --------------------------------------------------------------------------------------

def _torus_gaussian(w: int, h: int, sigma: float) -> np.ndarray:
    dy = np.minimum(np.arange(h), h - np.arange(h)).astype(np.float64)
    dx = np.minimum(np.arange(w), w - np.arange(w)).astype(np.float64)
    return np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2.0 * sigma * sigma))


@functools.lru_cache(maxsize=8)
def void_and_cluster(w: int, h: int, seed: int, sigma: float = 1.5) -> np.ndarray:
    """Void-and-cluster dither-array ranks (Ulichney 1993), shape (h, w), values 0..w*h-1.

    Energy is a Gaussian filter (sigma in pixels) on the torus; ties go to the lowest
    flat index (numpy argmax/argmin). The initial pattern marks 10% of the pixels, chosen
    by a seeded permutation.
    """
    n = w * h
    g = _torus_gaussian(w, h, sigma)

    def splat(y: int, x: int) -> np.ndarray:
        return np.roll(np.roll(g, y, axis=0), x, axis=1).ravel()

    order = np.argsort(splitmix64(seed, 0x7EE, n), kind="stable")
    n_init = max(1, n // 10)
    pattern = np.zeros(n, dtype=bool)
    pattern[order[:n_init]] = True
    energy = np.zeros(n)
    for p in np.flatnonzero(pattern):
        energy += splat(p // w, p % w)

    # Move points from the tightest cluster to the largest void until stable.
    for _ in range(10 * n):
        c = int(np.where(pattern, energy, -np.inf).argmax())
        pattern[c] = False
        energy -= splat(c // w, c % w)
        v = int(np.where(pattern, np.inf, energy).argmin())
        pattern[v] = True
        energy += splat(v // w, v % w)
        if v == c:
            break

    rank = np.full(n, -1, dtype=np.int64)
    # Phase 1: peel the initial pattern, tightest cluster first, ranks n_init-1 .. 0.
    p1, e1 = pattern.copy(), energy.copy()
    for r in range(n_init - 1, -1, -1):
        c = int(np.where(p1, e1, -np.inf).argmax())
        p1[c] = False
        e1 -= splat(c // w, c % w)
        rank[c] = r
    # Phase 2: fill the largest voids up to half the pixels.
    p2, e2 = pattern.copy(), energy.copy()
    r = n_init
    while r < n // 2:
        v = int(np.where(p2, np.inf, e2).argmin())
        p2[v] = True
        e2 += splat(v // w, v % w)
        rank[v] = r
        r += 1
    # Phase 3: the zeros are now the minority; remove their tightest clusters.
    e3 = np.zeros(n)
    for p in np.flatnonzero(~p2):
        e3 += splat(p // w, p % w)
    while r < n:
        c = int(np.where(~p2, e3, -np.inf).argmax())
        p2[c] = True
        e3 -= splat(c // w, c % w)
        rank[c] = r
        r += 1
    assert (rank >= 0).all()
    return rank.reshape(h, w)


def shift_tile(w: int, h: int, seed: int) -> np.ndarray:
    """uint32 Cranley-Patterson shifts, shape (h, w).

    The top log2(w*h) bits hold the void-and-cluster rank; the low bits are seeded
    uniform dither inside the rank's bin, so shifts cover all 32 bits while keeping
    the blue-noise ordering. Requires w*h to be a power of two.
    """
    n = w * h
    bits = n.bit_length() - 1
    if 1 << bits != n:
        raise ValueError("shift_tile needs w*h to be a power of two")
    rank = void_and_cluster(w, h, seed).astype(np.uint64).ravel()
    dither = splitmix64(seed, 0xD17, n) >> np.uint64(32 + bits)
    r = (rank << np.uint64(32 - bits)) | dither
    return r.astype(np.uint32).reshape(h, w)


def shift_tile_3d(w: int, h: int, d: int, seed: int) -> np.ndarray:
    """uint32 space-time shifts psi(j, n), shape (d, h, w): layer n of pixel p holds
    ((n + o(p)) mod d + (R(p) + u) / (w h)) / d in 32-bit fixed point.

    R is a void-and-cluster rank tile (blue noise in space) and o(p) in [0, d) the
    d-level quantisation of a second, independent rank tile; u is seeded uniform dither.
    Every pixel's d values fall in d distinct strata of [0, 1) (stratified in time), and
    every layer holds each stratum w h / d times. Requires d to divide w h.
    """
    n = w * h
    if d < 1 or n % d:
        raise ValueError("shift_tile_3d needs 1 <= d dividing w*h")
    rank = void_and_cluster(w, h, seed).astype(np.float64).ravel()
    off = (void_and_cluster(w, h, seed + 1).astype(np.int64).ravel() * d) // n
    u = uniform01(seed, 0x3D, n)
    fine = (rank + u) / n
    out = np.empty((d, n), dtype=np.uint32)
    for layer in range(d):
        stratum = (layer + off) % d
        v = (stratum + fine) / d
        out[layer] = np.minimum(np.floor(v * 4294967296.0), 4294967295.0).astype(np.uint32)
    return out.reshape(d, h, w)


def occluder_triangles(n_tri: int, seed: int, size: float = 0.01) -> np.ndarray:
    """Occluders for the connections' visibility: n_tri small triangles, shape (n_tri, 9)
    float32 (v0, v1, v2). Centres are uniform in [0, 1)^3; each vertex is the centre plus
    an isotropic normal offset of standard deviation `size`."""
    c = uniform01(seed, 0x7A1, 3 * n_tri).reshape(n_tri, 1, 3)
    off = normal(seed, 0x7A2, 9 * n_tri).reshape(n_tri, 3, 3) * size
    return (c + off).reshape(n_tri, 9).astype(np.float32)


# --------------------------------------------------------------------------------------
# Culling scale
# --------------------------------------------------------------------------------------

def calibrate_tau(light_pos: np.ndarray, intensity: np.ndarray, eye_pos: np.ndarray,
                  target: float, max_lights: int = 0) -> np.float32:
    """tau such that mean_j sum_i min(1, tau*I_i / max(|l_i - e_j|^2, 1e-4)) == target.

    Evaluated in float64 over the given eye sample (a workload-shaping step: the exact
    float32 rule that decides acceptance lives in the method, not here). Solved by
    bisection in log space over sorted per-pair ratios. With max_lights > 0, every k-th
    light stands for k lights (k = ceil(N_l / max_lights)).
    """
    stride = 1
    if max_lights and len(light_pos) > max_lights:
        stride = -(-len(light_pos) // max_lights)
    lp = light_pos[::stride].astype(np.float64)
    li = intensity[::stride].astype(np.float64)
    target = target / stride
    xs = []
    for e in eye_pos.astype(np.float64):
        d2 = ((lp - e) ** 2).sum(axis=1)
        xs.append(li / np.maximum(d2, 1e-4))
    x = np.sort(np.concatenate(xs))[::-1]  # descending
    csum = np.concatenate([[0.0], np.cumsum(x)])
    total = csum[-1]
    n_e = len(eye_pos)
    want = target * n_e

    def f(tau: float) -> float:
        # number of ratios >= 1/tau contribute 1 each, the rest tau*x
        k = int(np.searchsorted(-x, -1.0 / tau, side="right"))
        return k + tau * (total - csum[k])

    lo, hi = 1e-30, 1e30
    for _ in range(400):
        mid = math.sqrt(lo * hi)
        if f(mid) < want:
            lo = mid
        else:
            hi = mid
        if hi / lo < 1 + 1e-12:
            break
    return np.float32(math.sqrt(lo * hi))


# --------------------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------------------

class Scene(dict):
    """dict with keys: light_pos (N_l,3) f32, intensity (N_l,) f32, eye_pos (N_e,3) f32,
    px, py (N_e,) u16, tile (H,W) u32, tau f32, name str."""

    def __getattr__(self, k):
        try:
            return self[k]
        except KeyError as exc:  # pragma: no cover
            raise AttributeError(k) from exc


def _pixel_grid(w: int, h: int):
    py, px = np.divmod(np.arange(w * h, dtype=np.int64), w)
    return px.astype(np.uint16), py.astype(np.uint16)


def _eye_sample(n_e: int, k: int) -> np.ndarray:
    return np.unique(np.linspace(0, n_e - 1, num=min(k, n_e)).round().astype(np.int64))


@functools.lru_cache(maxsize=4)
def scene_uniform(n_lights: int = 4096, grid_w: int = 32, grid_h: int = 32,
                  tile_w: int = 32, tile_h: int = 32, target: float = 32.0,
                  sigma_i: float = 1.0, seed: int = 1) -> Scene:
    """Lights uniform in [0,1)^3 with lognormal(0, sigma_i) intensities; one eye per pixel
    of a grid_w x grid_h grid (eye j at pixel (j mod grid_w, j div grid_w)), positions
    uniform in [0,1)^3; a tile_w x tile_h shift tile; tau for ``target`` accepted/eye."""
    n_e = grid_w * grid_h
    light_pos = _to_unit_f32(uniform01(seed, 1, 3 * n_lights).reshape(n_lights, 3))
    intensity = np.exp(sigma_i * normal(seed, 2, n_lights)).astype(np.float32)
    eye_pos = _to_unit_f32(uniform01(seed, 3, 3 * n_e).reshape(n_e, 3))
    px, py = _pixel_grid(grid_w, grid_h)
    tile = shift_tile(tile_w, tile_h, seed)
    tau = calibrate_tau(light_pos, intensity, eye_pos[_eye_sample(n_e, 256)], target)
    return Scene(name=f"uniform_{n_e}x{n_lights}", light_pos=light_pos, intensity=intensity,
                 eye_pos=eye_pos, px=px, py=py, tile=tile, tau=tau)


def heightfield(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """The frame workload's eye surface: 0.5 + 0.25 sin(6 pi u) cos(4 pi v), in [0,1]."""
    return np.clip(0.5 + 0.25 * np.sin(6.0 * math.pi * u) * np.cos(4.0 * math.pi * v), 0.0, 1.0)


def gaussian_mixture_lights(n_lights: int, n_comp: int, seed: int,
                            sigma_lo: float = 0.02, sigma_hi: float = 0.1) -> np.ndarray:
    """n_lights points from n_comp isotropic Gaussians (centres U[0,1)^3, sigma
    U[sigma_lo, sigma_hi], uniform weights), rejecting samples outside [0,1)^3."""
    centres = uniform01(seed, 10, 3 * n_comp).reshape(n_comp, 3)
    sigmas = sigma_lo + (sigma_hi - sigma_lo) * uniform01(seed, 11, n_comp)
    out = []
    have = 0
    offset = 0
    while have < n_lights:
        batch = max(1024, 2 * (n_lights - have))
        comp = np.minimum((uniform01(seed, 12, batch, offset) * n_comp).astype(np.int64), n_comp - 1)
        z = normal(seed, 13, 3 * batch, 3 * offset).reshape(batch, 3)
        p = centres[comp] + sigmas[comp, None] * z
        ok = ((p >= 0.0) & (p < 1.0)).all(axis=1)
        out.append(p[ok])
        have += int(ok.sum())
        offset += batch
    return _to_unit_f32(np.concatenate(out)[:n_lights])


@functools.lru_cache(maxsize=4)
def scene_frame(width: int = 1920, height: int = 1080, n_lights: int = 1 << 20,
                tile_w: int = 64, tile_h: int = 64, target: float = 64.0,
                n_comp: int = 64, sigma_i: float = 1.5, seed: int = 2,
                tau_eyes: int = 32, tau_lights: int = 0) -> Scene:
    """Frame-sized workload: eye j at pixel (j mod width, j div width) with position
    (u, v, heightfield(u, v)), u = (px + U)/width, v = (py + U)/height; lights from a
    Gaussian mixture; lognormal(0, sigma_i) intensities; a tile_w x tile_h shift tile;
    tau for ``target`` accepted lights per eye (estimated on ``tau_eyes`` eyes)."""
    n_e = width * height
    px, py = _pixel_grid(width, height)
    ju = uniform01(seed, 20, 2 * n_e)
    u = (px.astype(np.float64) + ju[0::2]) / width
    v = (py.astype(np.float64) + ju[1::2]) / height
    eye_pos = _to_unit_f32(np.stack([u, v, heightfield(u, v)], axis=1))
    light_pos = gaussian_mixture_lights(n_lights, n_comp, seed)
    intensity = np.exp(sigma_i * normal(seed, 21, n_lights)).astype(np.float32)
    tile = shift_tile(tile_w, tile_h, seed)
    tau = calibrate_tau(light_pos, intensity, eye_pos[_eye_sample(n_e, tau_eyes)], target,
                        max_lights=tau_lights)
    return Scene(name=f"frame_{width}x{height}_{n_lights}", light_pos=light_pos,
                 intensity=intensity, eye_pos=eye_pos, px=px, py=py, tile=tile, tau=tau)


def rangemin_queries(n: int, seed: int = 3):
    """(a, b, r) uint32 triples: a uniform in [0, 2^32 - 1), len = floor(exp(U ln(2^32 - a)))
    clamped to [1, 2^32 - 1 - a] (log-uniform), b = a + len, r uniform in [0, 2^32)."""
    a = (splitmix64(seed, 30, n) % np.uint64(0xFFFFFFFF)).astype(np.uint64)
    span = (np.float64(2.0 ** 32) - a.astype(np.float64))
    ln = np.floor(np.exp(uniform01(seed, 31, n) * np.log(span)))
    ln = np.clip(ln, 1.0, (np.uint64(0xFFFFFFFF) - a).astype(np.float64)).astype(np.uint64)
    b = a + ln
    r = (splitmix64(seed, 32, n) >> np.uint64(32)).astype(np.uint32)
    return a.astype(np.uint32), b.astype(np.uint32), r


def log_uniform_int(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers log-uniform in [lo, hi]."""
    u = uniform01(seed, stream, n)
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))).astype(np.int64).clip(lo, hi)


def frame_sizes(n_frames: int = 64, seed: int = 4, eyes=(65536, 2073600), lights=(16384, 4194304),
                targets=(16.0, 128.0)):
    """Per-frame (width, height, n_lights, target) of the batched workload: N_e and N_l
    log-uniform in the given ranges (eyes laid out as a 16:9 frame of about N_e pixels),
    target accepted lights per eye uniform in ``targets``."""
    ne = log_uniform_int(seed, 40, n_frames, *eyes)
    nl = log_uniform_int(seed, 41, n_frames, *lights)
    tg = targets[0] + (targets[1] - targets[0]) * uniform01(seed, 42, n_frames)
    out = []
    for e, l_, t in zip(ne, nl, tg):
        w = max(1, int(round(math.sqrt(e * 16.0 / 9.0))))
        h = max(1, int(round(e / w)))
        out.append((w, h, int(l_), float(t)))
    return out


def batch_frames(n_frames: int = 64, seed: int = 4, **kw):
    """The batched workload: frames as in ``scene_frame`` with per-frame seeds, sizes and
    targets from ``frame_sizes`` (tau calibrated on a light subsample)."""
    frames = []
    for f, (w, h, n_l, t) in enumerate(frame_sizes(n_frames, seed, **kw)):
        frames.append(scene_frame.__wrapped__(width=w, height=h, n_lights=n_l, target=t,
                                              seed=1000 * seed + f, tau_eyes=16, tau_lights=65536))
    return frames
