"""Python access to the CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg, never by the product package. The oracle is plain C built
with gcc (``-ffp-contract=off -frounding-math``) and shares nothing with the CUDA library
except the seeded inputs from ``synth``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-frounding-math",
          "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas"]


def build(force: bool = False, openmp: bool = True, out: str | None = None) -> str:
    """Compile ``liboracle.so`` (with OpenMP when asked for and the compiler has it; the
    plain C99 build without it is single-threaded). ``out`` names another library file."""
    lib_path = out or _LIB
    os.makedirs(os.path.dirname(lib_path), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= newest:
        return lib_path
    tmp = lib_path + f".tmp{os.getpid()}"
    base = ["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"]
    if openmp:
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
    else:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, lib_path)
    return lib_path


class _Result(C.Structure):
    _fields_ = [
        ("n_pairs", C.c_uint64),
        ("pairs", C.POINTER(C.c_uint32)),
        ("count", C.POINTER(C.c_uint32)),
        ("visits", C.POINTER(C.c_uint64)),
        ("total_visits", C.c_uint64),
        ("n_marginal", C.c_uint64),
        ("seconds", C.c_double),
        ("threads", C.c_int),
    ]


class _Tree(C.Structure):
    _fields_ = [
        ("n", C.c_uint32),
        ("height", C.c_uint32),
        ("perm", C.POINTER(C.c_uint32)),
        ("key", C.POINTER(C.c_uint64)),
        ("pos", C.POINTER(C.c_float)),
        ("inten", C.POINTER(C.c_float)),
        ("first", C.POINTER(C.c_uint32)),
        ("last", C.POINTER(C.c_uint32)),
        ("split", C.POINTER(C.c_uint32)),
        ("lo", C.POINTER(C.c_float)),
        ("hi", C.POINTER(C.c_float)),
        ("imax", C.POINTER(C.c_float)),
    ]


def configure(L):
    """Set the argument and result types of an oracle library's functions (any build)."""
    u32, u64, f32, i32 = C.c_uint32, C.c_uint64, C.c_float, C.c_int
    P = C.c_void_p
    L.or_brev.restype = u32
    L.or_brev.argtypes = [u32, i32]
    for nm in ("or_rangemin_scan", "or_rangemin_trie"):
        getattr(L, nm).restype = u32
        getattr(L, nm).argtypes = [u64, u64, u32, i32, C.POINTER(u64)]
    L.or_alg1.restype = u64
    L.or_alg1.argtypes = [u64, u64, i32]
    for nm in ("or_alg2_printed", "or_alg2_fixed"):
        getattr(L, nm).restype = u64
        getattr(L, nm).argtypes = [u64, u64, u32, i32]
    L.or_rangemin_batch.restype = None
    L.or_rangemin_batch.argtypes = [P, P, P, u64, i32, i32, P, P, i32]
    L.or_fround.restype = f32
    L.or_fround.argtypes = [i32, f32, f32, i32]
    L.or_fma_rd.restype = f32
    L.or_fma_rd.argtypes = [f32, f32, f32]
    L.or_leaf_threshold.restype = u64
    L.or_leaf_threshold.argtypes = [f32, P, f32, P]
    L.or_node_culls.restype = i32
    L.or_node_culls.argtypes = [f32, P, P, f32, P, u32]
    L.or_morton.restype = u64
    L.or_morton.argtypes = [f32, f32, f32]
    L.or_tree_build.restype = C.POINTER(_Tree)
    L.or_tree_build.argtypes = [P, P, u32]
    L.or_tree_build_cost.restype = C.POINTER(_Tree)
    L.or_tree_build_cost.argtypes = [P, P, u32, u32]
    L.or_tree_free.restype = None
    L.or_tree_free.argtypes = [C.POINTER(_Tree)]
    L.or_tree_refit.restype = None
    L.or_tree_refit.argtypes = [C.POINTER(_Tree), P, P]
    for nm in ("or_cull_flat", "or_cull_hier"):
        getattr(L, nm).restype = C.POINTER(_Result)
        getattr(L, nm).argtypes = [C.POINTER(_Tree), P, P, P, P, u32, P, u32, u32, f32, i32]
    L.or_cull_hier_w.restype = C.POINTER(_Result)
    L.or_cull_hier_w.argtypes = [C.POINTER(_Tree), P, P, P, P, u32, P, u32, u32, f32, i32, i32]
    L.or_cull_free.restype = None
    L.or_cull_free.argtypes = [C.POINTER(_Result)]
    L.or_max_threads.restype = i32
    L.or_pair_weight.restype = None
    L.or_pair_weight.argtypes = [f32, P, f32, P, P, P]
    L.or_segment_hits.restype = i32
    L.or_segment_hits.argtypes = [P, P, P]
    L.or_connect.restype = None
    L.or_connect.argtypes = [P, u32, P, P, P, u64, f32, P, u32, P, P, P, i32]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = configure(C.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---- range minimum ---------------------------------------------------------------------

def brev(x: int, B: int = 32) -> int:
    return int(lib().or_brev(x, B))


def rangemin_scan(a: int, b: int, r: int, B: int = 32):
    k = C.c_uint64()
    v = lib().or_rangemin_scan(a, b, r, B, C.byref(k))
    return int(v), int(k.value)


def rangemin_trie(a: int, b: int, r: int, B: int = 32):
    k = C.c_uint64()
    v = lib().or_rangemin_trie(a, b, r, B, C.byref(k))
    return int(v), int(k.value)


def alg1(a: int, b: int, B: int = 32) -> int:
    return int(lib().or_alg1(a, b, B))


def alg2_printed(a: int, b: int, r: int, B: int = 32) -> int:
    return int(lib().or_alg2_printed(a, b, r, B))


def alg2_fixed(a: int, b: int, r: int, B: int = 32) -> int:
    return int(lib().or_alg2_fixed(a, b, r, B))


METHODS = {"scan": 0, "trie": 1, "alg2": 2, "alg2_printed": 3, "alg1": 4, "scan_inc": 5}


def rangemin_batch(a, b, r, method: str = "trie", nthreads: int = 0, want_argmin: bool = True,
                   B: int = 32):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    n = len(a)
    v = np.empty(n, dtype=np.uint32)
    k = np.empty(n, dtype=np.uint32) if want_argmin else None
    lib().or_rangemin_batch(_ptr(a), _ptr(b), _ptr(r), n, METHODS[method], B, _ptr(v),
                            _ptr(k) if k is not None else None, nthreads)
    return v, k


# ---- thresholds --------------------------------------------------------------------------

def fround(op: str, x: float, y: float, mode: int) -> np.float32:
    ops = {"add": 0, "sub": 1, "mul": 2, "div": 3}
    return np.float32(lib().or_fround(ops[op], np.float32(x), np.float32(y), mode))


def fma_rd(x: float, y: float, z: float) -> np.float32:
    """x y + z rounded once toward -inf, in float32."""
    return np.float32(lib().or_fma_rd(np.float32(x), np.float32(y), np.float32(z)))


def leaf_threshold(tau, l, intensity, e) -> int:
    l = np.ascontiguousarray(l, dtype=np.float32)
    e = np.ascontiguousarray(e, dtype=np.float32)
    return int(lib().or_leaf_threshold(np.float32(tau), _ptr(l), np.float32(intensity), _ptr(e)))


def node_culls(tau, lo, hi, imax, e, v) -> bool:
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    e = np.ascontiguousarray(e, dtype=np.float32)
    return bool(lib().or_node_culls(np.float32(tau), _ptr(lo), _ptr(hi), np.float32(imax), _ptr(e), int(v)))


def node_cull_floor(tau, lo, hi, imax, e) -> int:
    """Smallest v in [0, 2^32] for which the node culls (2^32: never), by bisection (the
    test is monotone in v)."""
    if not node_culls(tau, lo, hi, imax, e, 0xFFFFFFFF):
        return 1 << 32
    if node_culls(tau, lo, hi, imax, e, 0):
        return 0
    lo_v, hi_v = 0, 0xFFFFFFFF  # culls(hi_v) holds, culls(lo_v) does not
    while hi_v - lo_v > 1:
        mid = (lo_v + hi_v) // 2
        if node_culls(tau, lo, hi, imax, e, mid):
            hi_v = mid
        else:
            lo_v = mid
    return hi_v


def morton(x, y, z) -> int:
    return int(lib().or_morton(np.float32(x), np.float32(y), np.float32(z)))


# ---- hierarchy and culling -----------------------------------------------------------------

class Tree:
    """Oracle light hierarchy: Morton-sorted leaves and a top-down binary radix tree."""

    def __init__(self, light_pos: np.ndarray, intensity: np.ndarray, topology: str = "radix", cost_depth: int = 0):
        self._pos = np.ascontiguousarray(light_pos, dtype=np.float32).reshape(-1, 3)
        self._inten = np.ascontiguousarray(intensity, dtype=np.float32)
        self.n = len(self._inten)
        if topology == "radix":
            self._t = lib().or_tree_build(_ptr(self._pos), _ptr(self._inten), self.n)
        elif topology == "cost":
            self._t = lib().or_tree_build_cost(_ptr(self._pos), _ptr(self._inten), self.n, cost_depth)
        else:
            raise ValueError(f"unknown topology {topology!r}")
        if not self._t:
            raise ValueError("empty light set")
        t = self._t.contents
        n, ni = self.n, self.n - 1
        self.height = int(t.height)
        self.perm = np.ctypeslib.as_array(t.perm, shape=(n,)).copy()
        self.key = np.ctypeslib.as_array(t.key, shape=(n,)).copy()
        self.pos = np.ctypeslib.as_array(t.pos, shape=(n * 3,)).reshape(n, 3).copy()
        self.inten = np.ctypeslib.as_array(t.inten, shape=(n,)).copy()
        if ni:
            self.first = np.ctypeslib.as_array(t.first, shape=(ni,)).copy()
            self.last = np.ctypeslib.as_array(t.last, shape=(ni,)).copy()
            self.split = np.ctypeslib.as_array(t.split, shape=(ni,)).copy()
            self.lo = np.ctypeslib.as_array(t.lo, shape=(ni * 3,)).reshape(ni, 3).copy()
            self.hi = np.ctypeslib.as_array(t.hi, shape=(ni * 3,)).reshape(ni, 3).copy()
            self.imax = np.ctypeslib.as_array(t.imax, shape=(ni,)).copy()
        else:
            e32 = np.zeros(0, dtype=np.uint32)
            self.first = self.last = self.split = e32
            self.lo = self.hi = np.zeros((0, 3), dtype=np.float32)
            self.imax = np.zeros(0, dtype=np.float32)

    def _read_boxes(self):
        t = self._t.contents
        n, ni = self.n, self.n - 1
        self.pos = np.ctypeslib.as_array(t.pos, shape=(n * 3,)).reshape(n, 3).copy()
        self.inten = np.ctypeslib.as_array(t.inten, shape=(n,)).copy()
        if ni:
            self.lo = np.ctypeslib.as_array(t.lo, shape=(ni * 3,)).reshape(ni, 3).copy()
            self.hi = np.ctypeslib.as_array(t.hi, shape=(ni * 3,)).reshape(ni, 3).copy()
            self.imax = np.ctypeslib.as_array(t.imax, shape=(ni,)).copy()

    def refit(self, light_pos: np.ndarray, intensity: np.ndarray):
        """Moved lights (same ids): keep the leaf order and topology, recompute the boxes
        and maximum intensities from the new positions."""
        pos = np.ascontiguousarray(light_pos, dtype=np.float32).reshape(-1, 3)
        inten = np.ascontiguousarray(intensity, dtype=np.float32)
        if len(inten) != self.n or len(pos) != self.n:
            raise ValueError("refit needs the same number of lights")
        self._pos, self._inten = pos, inten
        lib().or_tree_refit(self._t, _ptr(pos), _ptr(inten))
        self._read_boxes()

    def __del__(self):
        t = getattr(self, "_t", None)
        if t:
            lib().or_tree_free(t)
            self._t = None


def spacetime_layer(tile, sample_index: int = 0) -> np.ndarray:
    """The shifts of sample n: a (h, w) tile is used as is; a (d, h, w) space-time tile
    psi(j, n) (Sec. 3, the 3D-tile option) gives layer n mod d."""
    tile = np.asarray(tile, dtype=np.uint32)
    if tile.ndim == 3:
        return tile[int(sample_index) % tile.shape[0]]
    return tile


def _cull(fn, tree: Tree, eye_pos, px, py, tile, tau, eye_ids=None, nthreads=0, sample_index=0, width=None):
    eye_pos = np.ascontiguousarray(eye_pos, dtype=np.float32).reshape(-1, 3)
    px = np.ascontiguousarray(px, dtype=np.uint16)
    py = np.ascontiguousarray(py, dtype=np.uint16)
    tile = np.ascontiguousarray(spacetime_layer(tile, sample_index), dtype=np.uint32)
    h, w = tile.shape
    ids = None if eye_ids is None else np.ascontiguousarray(eye_ids, dtype=np.uint32)
    n_e = len(eye_pos)
    extra = () if width is None else (int(width),)
    res = fn(tree._t, _ptr(eye_pos), _ptr(px), _ptr(py), _ptr(ids) if ids is not None else None,
             n_e, _ptr(tile), w, h, np.float32(tau), *extra, nthreads)
    try:
        r = res.contents
        n = int(r.n_pairs)
        out = {
            "pairs": np.ctypeslib.as_array(r.pairs, shape=(2 * n,)).reshape(n, 2).copy() if n
            else np.zeros((0, 2), dtype=np.uint32),
            "count": np.ctypeslib.as_array(r.count, shape=(n_e,)).copy() if n_e
            else np.zeros(0, dtype=np.uint32),
            "visits": np.ctypeslib.as_array(r.visits, shape=(n_e,)).copy() if (r.visits and n_e)
            else None,
            "total_visits": int(r.total_visits),
            "n_marginal": int(r.n_marginal),
            "seconds": float(r.seconds),
            "threads": int(r.threads),
        }
    finally:
        lib().or_cull_free(res)
    return out


def cull_flat(tree: Tree, eye_pos, px, py, tile, tau, eye_ids=None, nthreads=0, sample_index=0):
    """Every (eye, light) pair tested: the definition of the accepted set."""
    return _cull(lib().or_cull_flat, tree, eye_pos, px, py, tile, tau, eye_ids, nthreads, sample_index)


def cull_hier(tree: Tree, eye_pos, px, py, tile, tau, eye_ids=None, nthreads=0, sample_index=0, width=2):
    """Hierarchical traversal with per-eye visit counts; must equal ``cull_flat``. width 2
    visits binary nodes; width 4 visits the tree as nodes of width four (even depths,
    grandchildren tested), with visits counted per such node."""
    if width not in (2, 4):
        raise ValueError("width must be 2 or 4")
    return _cull(lib().or_cull_hier_w, tree, eye_pos, px, py, tile, tau, eye_ids, nthreads, sample_index,
                 width=width)


def max_threads() -> int:
    return int(lib().or_max_threads())


# ---- connection evaluation ----------------------------------------------------------

def pair_weight(tau, l, intensity, e):
    """(weight, p) of one accepted connection: (I / max(d^2, 1e-4)) / p in float32."""
    lv = np.ascontiguousarray(l, dtype=np.float32)
    ev = np.ascontiguousarray(e, dtype=np.float32)
    w, p = C.c_float(), C.c_float()
    lib().or_pair_weight(np.float32(tau), _ptr(lv), np.float32(intensity), _ptr(ev), C.byref(w), C.byref(p))
    return np.float32(w.value), np.float32(p.value)


def segment_hits(e, l, tri) -> bool:
    """Whether the open segment e -> l crosses the closed triangle (3 x 3 vertices)."""
    ev = np.ascontiguousarray(e, dtype=np.float32)
    lv = np.ascontiguousarray(l, dtype=np.float32)
    tv = np.ascontiguousarray(tri, dtype=np.float32).reshape(9)
    return bool(lib().or_segment_hits(_ptr(ev), _ptr(lv), _ptr(tv)))


def connect(eye_pos, light_pos, intensity, pairs, tau, tris=None, nthreads=0):
    """Per accepted pair (eye id, light id): weight x visibility (float32), visibility,
    and per-eye sums (float64). light_pos / intensity are indexed by light id."""
    eye_pos = np.ascontiguousarray(eye_pos, dtype=np.float32).reshape(-1, 3)
    light_pos = np.ascontiguousarray(light_pos, dtype=np.float32).reshape(-1, 3)
    intensity = np.ascontiguousarray(intensity, dtype=np.float32)
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    tris = np.zeros((0, 9), np.float32) if tris is None else np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    n = len(pairs)
    weight = np.zeros(max(n, 1), np.float32)
    vis = np.zeros(max(n, 1), np.uint8)
    sums = np.zeros(max(len(eye_pos), 1), np.float64)
    lib().or_connect(_ptr(eye_pos), len(eye_pos), _ptr(light_pos), _ptr(intensity), _ptr(pairs), n,
                     np.float32(tau), _ptr(tris), len(tris), _ptr(weight), _ptr(vis), _ptr(sums), nthreads)
    return {"weight": weight[:n], "visible": vis[:n].astype(bool), "eye_sum": sums[:len(eye_pos)]}
