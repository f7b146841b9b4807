"""Python binding of ``libhrr`` (blue-noise dithered QMC hierarchical Russian roulette).

A thin ctypes layer over the C ABI declared in ``include/hrr.h``: the functions below have
the C names and only marshal arguments (device pointers of PyTorch CUDA tensors, sizes,
handles). Every step of the culling path runs in the library's sm_103a kernels; there is
no CPU fallback, and importing this module raises if the library has not been built.

``Context`` wraps a context handle for callers holding PyTorch tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhrr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = C.CDLL(LIB_PATH)

HRR_OK = 0
HRR_ERR_INVALID_ARG = 1
HRR_ERR_OOM = 2
HRR_ERR_NO_TILE = 3
HRR_ERR_OVERFLOW = 4
HRR_ERR_TIMEOUT = 5
HRR_ERR_CUDA = 6
HRR_ERR_DEVICE = 7
HRR_PENDING = 8


class hrr_lights(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("intensity", C.c_void_p)]


class hrr_eyes(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("px", C.c_void_p), ("py", C.c_void_p)]


class hrr_node(C.Structure):
    _fields_ = [("c0_lo", C.c_float * 3), ("c0_imax", C.c_float),
                ("c0_hi", C.c_float * 3), ("split", C.c_uint32),
                ("c1_lo", C.c_float * 3), ("c1_imax", C.c_float),
                ("c1_hi", C.c_float * 3), ("other_end", C.c_uint32)]


assert C.sizeof(hrr_node) == 64

NODE_DTYPE = np.dtype([("c0_lo", "<f4", 3), ("c0_imax", "<f4"), ("c0_hi", "<f4", 3),
                       ("split", "<u4"), ("c1_lo", "<f4", 3), ("c1_imax", "<f4"),
                       ("c1_hi", "<f4", 3), ("other_end", "<u4")])


class hrr_frame(C.Structure):
    _fields_ = [("eyes", hrr_eyes), ("n_eyes", C.c_uint32), ("tree", C.c_void_p),
                ("dev_tile", C.c_void_p), ("tile_w", C.c_uint32), ("tile_h", C.c_uint32),
                ("tau", C.c_float), ("shift_offset", C.c_uint32), ("dev_pairs", C.c_void_p),
                ("cap", C.c_uint64), ("eye_visits", C.c_void_p), ("tile_d", C.c_uint32),
                ("sample_index", C.c_uint32)]


class hrr_job(C.Structure):
    _fields_ = [("eyes", hrr_eyes), ("n_eyes", C.c_uint32), ("tree", C.c_void_p),
                ("dev_tile", C.c_void_p), ("tile_w", C.c_uint32), ("tile_h", C.c_uint32),
                ("tau", C.c_float), ("shift_offset", C.c_uint32), ("cap", C.c_uint64),
                ("tile_d", C.c_uint32), ("sample_index", C.c_uint32), ("refit", hrr_lights)]


class hrr_job_result(C.Structure):
    _fields_ = [("status", C.c_int), ("count", C.c_uint64), ("visits", C.c_uint64),
                ("dev_pairs", C.c_void_p), ("queue_s", C.c_double), ("latency_s", C.c_double)]


class hrr_server_info(C.Structure):
    _fields_ = [("slices", C.c_uint64), ("launches", C.c_uint64), ("jobs_done", C.c_uint64),
                ("jobs_waiting", C.c_uint64), ("jobs_active", C.c_uint64),
                ("bytes_reserved", C.c_uint64), ("max_active", C.c_uint32)]


class hrr_cull_opts(C.Structure):
    _fields_ = [("eye_visits", C.c_void_p), ("rangemin_variant", C.c_int),
                ("shift_offset", C.c_uint32), ("blocks_per_sm", C.c_uint32),
                ("sample_index", C.c_uint32), ("node_width", C.c_uint32),
                ("ring_entries", C.c_uint32), ("threads_per_block", C.c_uint32),
                ("top_levels", C.c_uint32)]


class hrr_peaks(C.Structure):
    _fields_ = [("l2_read_gbs", C.c_double), ("record_fetches_per_s", C.c_double), ("int_ops_per_s", C.c_double)]


class hrr_build_opts(C.Structure):
    _fields_ = [("topology", C.c_int), ("cost_depth", C.c_uint32)]


HRR_TOPOLOGY_RADIX, HRR_TOPOLOGY_COST = 0, 1
TOPOLOGIES = {"radix": HRR_TOPOLOGY_RADIX, "cost": HRR_TOPOLOGY_COST}


TUNING_FIELDS = ("rangemin_variant", "blocks_per_sm", "node_width", "ring_entries", "threads_per_block",
                 "top_levels")


class hrr_tuning(C.Structure):
    _fields_ = [("rangemin_variant", C.c_int), ("blocks_per_sm", C.c_uint32), ("node_width", C.c_uint32),
                ("ring_entries", C.c_uint32), ("threads_per_block", C.c_uint32), ("top_levels", C.c_uint32)]

    @classmethod
    def from_dict(cls, d):
        if d is None:
            return None
        return cls(*(int(d.get(k, 0)) for k in TUNING_FIELDS))

    def to_dict(self):
        return {k: int(getattr(self, k)) for k in TUNING_FIELDS}


def _opts(eye_visits, tuning, rangemin_variant, shift_offset, sample_index):
    """hrr_cull_opts from a tuning dict (its fields win) and the call's own arguments."""
    t = tuning or {}
    return hrr_cull_opts(_ptr(eye_visits), int(t.get("rangemin_variant", rangemin_variant)), int(shift_offset),
                         int(t.get("blocks_per_sm", 0)), int(sample_index), int(t.get("node_width", 0)),
                         int(t.get("ring_entries", 0)), int(t.get("threads_per_block", 0)),
                         int(t.get("top_levels", 0)))


_P = C.c_void_p
_u32, _u64, _i32, _f32 = C.c_uint32, C.c_uint64, C.c_int, C.c_float
_SIGS = {
    "hrr_create": (_i32, [C.POINTER(_P), _i32, _P]),
    "hrr_destroy": (_i32, [_P]),
    "hrr_last_error": (C.c_char_p, [_P]),
    "hrr_status_string": (C.c_char_p, [_i32]),
    "hrr_launch_count": (_i32, [_P, C.POINTER(_u64)]),
    "hrr_set_timing": (_i32, [_P, _i32]),
    "hrr_kernel_time": (_i32, [_P, C.POINTER(C.c_double), C.POINTER(_u64)]),
    "hrr_build_light_tree": (_i32, [_P, hrr_lights, _u32, C.POINTER(_P)]),
    "hrr_free_light_tree": (_i32, [_P, _P]),
    "hrr_tree_perm": (_i32, [_P, C.POINTER(_P)]),
    "hrr_tree_info": (_i32, [_P, C.POINTER(_u32), C.POINTER(_u32), C.POINTER(_P)]),
    "hrr_tree_download": (_i32, [_P, _P, _P, _P]),
    "hrr_set_shift_tile": (_i32, [_P, _P, _u32, _u32]),
    "hrr_set_shift_tile_3d": (_i32, [_P, _P, _u32, _u32, _u32]),
    "hrr_refit_light_tree": (_i32, [_P, _P, hrr_lights]),
    "hrr_build_light_tree_ex": (_i32, [_P, hrr_lights, _u32, C.POINTER(hrr_build_opts), C.POINTER(_P)]),
    "hrr_build_light_tree_host": (_i32, [_P, hrr_lights, _u32, C.POINTER(hrr_build_opts), C.POINTER(_P)]),
    "hrr_build_scene": (_i32, [_P, _P, _u32, C.POINTER(_P)]),
    "hrr_free_scene": (_i32, [_P, _P]),
    "hrr_connect": (_i32, [_P, hrr_eyes, _u32, hrr_lights, _u32, _f32, _P, _u64, _P, _P, _P, _P]),
    "hrr_cull": (_i32, [_P, hrr_eyes, _u32, _P, _f32, _P, _u64, C.POINTER(_u64)]),
    "hrr_cull_ex": (_i32, [_P, hrr_eyes, _u32, _P, _f32, C.POINTER(hrr_cull_opts), _P, _u64,
                           C.POINTER(_u64)]),
    "hrr_cull_host": (_i32, [_P, hrr_eyes, _u32, _P, _f32, C.POINTER(hrr_cull_opts), _P, _u64,
                             C.POINTER(_u64)]),
    "hrr_last_cull_stats": (_i32, [_P, C.POINTER(_u64), C.POINTER(_u64)]),
    "hrr_measure_peaks": (_i32, [_P, C.POINTER(hrr_peaks)]),
    "hrr_cull_samples": (_i32, [_P, hrr_eyes, _u32, _P, _f32, _P, _u32, _P, _u64, _P, _P]),
    "hrr_range_min": (_i32, [_P, _P, _P, _P, _P, _P, _u64, _i32]),
    "hrr_build_light_tree_static": (_i32, [hrr_lights, _u32, _P, _P, C.POINTER(_u32), _P,
                                           C.c_char_p, C.c_size_t]),
    "hrr_batch_create": (_i32, [_P, C.POINTER(hrr_frame), _u32, C.POINTER(hrr_tuning), _i32, C.POINTER(_P)]),
    "hrr_batch_launch": (_i32, [_P, _P]),
    "hrr_batch_results": (_i32, [_P, _P, C.POINTER(_u64), C.POINTER(_u64)]),
    "hrr_batch_destroy": (_i32, [_P, _P]),
    "hrr_cull_batch": (_i32, [_P, C.POINTER(hrr_frame), _u32, C.POINTER(hrr_tuning), C.POINTER(_u64)]),
    "hrr_server_create": (_i32, [_P, _u64, _u32, _u32, C.POINTER(hrr_tuning), C.POINTER(_P)]),
    "hrr_autotune": (_i32, [_P, hrr_eyes, _u32, _P, _f32, _P, _u64, C.POINTER(hrr_tuning),
                            C.POINTER(C.c_double)]),
    "hrr_default_tuning": (_i32, [C.POINTER(hrr_tuning)]),
    "hrr_autotune_all": (_i32, [_P, hrr_eyes, _u32, _P, _f32, _P, _u64, C.POINTER(hrr_tuning),
                                C.POINTER(C.c_double), _u32, C.POINTER(_u32)]),
    "hrr_server_submit": (_i32, [_P, _P, C.POINTER(hrr_job), C.POINTER(_u64)]),
    "hrr_server_poll": (_i32, [_P, _u64, C.POINTER(hrr_job_result)]),
    "hrr_server_wait": (_i32, [_P, _u64, C.c_double, C.POINTER(hrr_job_result)]),
    "hrr_server_release": (_i32, [_P, _u64]),
    "hrr_server_stats": (_i32, [_P, C.POINTER(hrr_server_info)]),
    "hrr_server_destroy": (_i32, [_P]),
    "hrr_server_copy_pairs": (_i32, [_P, _u64, _P, _u64, C.POINTER(_u64)]),
}
STATIC_BUILD_MAX_LIGHTS = 65536
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


def default_tuning() -> dict:
    """The tuning the library uses for zero fields (hrr_default_tuning)."""
    t = hrr_tuning()
    hrr_default_tuning(C.byref(t))
    return t.to_dict()


class HRRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{hrr_status_string(status).decode()}: {msg}")
        self.status = status


def _ptr(t):
    """Device (or host) address of a tensor / array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _tile_dims(tile):
    """(d, h, w) of a device tile tensor of shape (h, w) or (d, h, w); zeros for None."""
    if tile is None:
        return 0, 0, 0
    if tile.dim() == 3:
        return int(tile.shape[0]), int(tile.shape[1]), int(tile.shape[2])
    return 1, int(tile.shape[0]), int(tile.shape[1])


class Context:
    """A library context bound to a CUDA device and stream (PyTorch's current stream by
    default). Methods take PyTorch CUDA tensors and return library handles / counts."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = _P()
        st = hrr_create(C.byref(h), device, _P(stream.cuda_stream))
        if st != HRR_OK:
            raise HRRError(st, "hrr_create")
        self.handle = h

    def check(self, st: int):
        if st != HRR_OK:
            raise HRRError(st, hrr_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            hrr_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    # -- shifts ----------------------------------------------------------------------------
    def set_shift_tile(self, tile: np.ndarray):
        """A (h, w) tile of shifts, or a (d, h, w) space-time tile (layer n mod d for
        sample index n)."""
        tile = np.ascontiguousarray(tile, dtype=np.uint32)
        if tile.ndim == 3:
            d, h, w = tile.shape
            self.check(hrr_set_shift_tile_3d(self.handle, tile.ctypes.data, w, h, d))
        else:
            h, w = tile.shape
            self.check(hrr_set_shift_tile(self.handle, tile.ctypes.data, w, h))

    # -- hierarchy -------------------------------------------------------------------------
    def build_light_tree(self, x, y, z, intensity, topology: str = "radix", cost_depth: int = 0) -> "Tree":
        """Hierarchy over the lights; topology "radix" (binary radix tree) or "cost"
        (cost-driven splits over the same leaf order down to depth ``cost_depth``, 0 = 48)."""
        n = int(x.numel())
        L = hrr_lights(_ptr(x), _ptr(y), _ptr(z), _ptr(intensity))
        t = _P()
        opts = hrr_build_opts(TOPOLOGIES[topology], cost_depth)
        self.check(hrr_build_light_tree_ex(self.handle, L, n, C.byref(opts), C.byref(t)))
        return Tree(self, t)

    def build_light_tree_host(self, x, y, z, intensity, topology: str = "radix", cost_depth: int = 0) -> "Tree":
        """build_light_tree from host arrays (numpy arrays or CPU tensors; pinned memory
        copies fastest): the library stages them on the device itself."""
        n = int(x.numel() if hasattr(x, "numel") else x.size)
        L = hrr_lights(_ptr(x), _ptr(y), _ptr(z), _ptr(intensity))
        t = _P()
        opts = hrr_build_opts(TOPOLOGIES[topology], cost_depth)
        self.check(hrr_build_light_tree_host(self.handle, L, n, C.byref(opts), C.byref(t)))
        return Tree(self, t)

    def refit_light_tree(self, tree: "Tree", x, y, z, intensity):
        """Refit ``tree`` in place to moved lights (same ids, same count)."""
        if int(x.numel()) != tree.n_lights:
            raise ValueError("refit needs the tree's light count")
        self.check(hrr_refit_light_tree(self.handle, tree.handle, hrr_lights(_ptr(x), _ptr(y), _ptr(z),
                                                                             _ptr(intensity))))

    # -- connection evaluation -------------------------------------------------------------
    def build_scene(self, tris) -> "Scene":
        """Triangle hierarchy from a (n, 9) float32 CUDA tensor (v0, v1, v2 per row)."""
        h = _P()
        self.check(hrr_build_scene(self.handle, _ptr(tris), int(tris.shape[0]), C.byref(h)))
        return Scene(self, h)

    def connect(self, x, y, z, lights, tau: float, pairs, n_pairs: int, scene=None, weight=None, visible=None,
                eye_sum=None):
        """Weights x visibility of the first n_pairs accepted pairs; lights = (x, y, z,
        intensity) tensors by light id; eye_sum (float32, one per eye) receives the sums."""
        E = hrr_eyes(_ptr(x), _ptr(y), _ptr(z), None, None)
        L = hrr_lights(*(_ptr(a) for a in lights))
        self.check(hrr_connect(self.handle, E, int(x.numel()), L, int(lights[0].numel()), float(tau), _ptr(pairs),
                               int(n_pairs), scene.handle if scene is not None else None, _ptr(weight),
                               _ptr(visible), _ptr(eye_sum)))

    # -- culling ---------------------------------------------------------------------------
    def cull(self, x, y, z, px, py, tree: "Tree", tau: float, pairs, eye_visits=None,
             rangemin_variant: int = 0, shift_offset: int = 0, tuning=None, sample_index: int = 0):
        """Cull into ``pairs`` (uint32/int32 tensor of shape (cap, 2)); returns
        (status, count). HRR_ERR_OVERFLOW is returned, not raised. ``tuning`` (a dict as
        returned by autotune) sets the launch shape and overrides rangemin_variant."""
        n = int(x.numel())
        E = hrr_eyes(_ptr(x), _ptr(y), _ptr(z), _ptr(px), _ptr(py))
        cap = int(pairs.shape[0]) if pairs is not None else 0
        cnt = _u64()
        opts = _opts(eye_visits, tuning, rangemin_variant, shift_offset, sample_index)
        st = hrr_cull_ex(self.handle, E, n, tree.handle, float(tau), C.byref(opts),
                         _ptr(pairs) if cap else None, cap, C.byref(cnt))
        if st not in (HRR_OK, HRR_ERR_OVERFLOW):
            self.check(st)
        return st, int(cnt.value)

    def cull_host(self, x, y, z, px, py, tree: "Tree", tau: float, pairs, rangemin_variant: int = 0,
                  shift_offset: int = 0, tuning=None, sample_index: int = 0):
        """``cull`` with host buffers: the eye arrays and ``pairs`` (shape (cap, 2), uint32 or
        int32) live in host memory (pinned memory lets the copies overlap the culling);
        returns (status, count)."""
        n = int(x.numel() if hasattr(x, "numel") else x.size)
        E = hrr_eyes(_ptr(x), _ptr(y), _ptr(z), _ptr(px), _ptr(py))
        cap = int(pairs.shape[0]) if pairs is not None else 0
        cnt = _u64()
        opts = _opts(None, tuning, rangemin_variant, shift_offset, sample_index)
        st = hrr_cull_host(self.handle, E, n, tree.handle, float(tau), C.byref(opts),
                           _ptr(pairs) if cap else None, cap, C.byref(cnt))
        if st not in (HRR_OK, HRR_ERR_OVERFLOW):
            self.check(st)
        return st, int(cnt.value)

    def cull_samples(self, x, y, z, px, py, tree: "Tree", tau: float, offsets, pairs):
        """Several samples per light in one traversal: sample s uses the shift offset
        offsets[s] (and layer s mod d of a space-time tile); ``pairs`` has shape
        (n_samples, cap, 2). Returns (status, counts per sample, (sample visits, records
        fetched)). HRR_ERR_OVERFLOW is returned, not raised."""
        import numpy as np
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64) & 0xFFFFFFFF, dtype=np.uint32)
        ns = int(off.size)
        cap = int(pairs.shape[1]) if pairs is not None and pairs.ndim == 3 else 0
        counts = np.zeros(max(ns, 1), np.uint64)
        visits = np.zeros(2, np.uint64)
        E = hrr_eyes(_ptr(x), _ptr(y), _ptr(z), _ptr(px), _ptr(py))
        st = hrr_cull_samples(self.handle, E, int(x.numel()), tree.handle, float(tau), off.ctypes.data, ns,
                              _ptr(pairs) if cap else None, cap, counts.ctypes.data, visits.ctypes.data)
        if st not in (HRR_OK, HRR_ERR_OVERFLOW):
            self.check(st)
        return st, [int(c) for c in counts[:ns]], (int(visits[0]), int(visits[1]))

    def measure_peaks(self) -> dict:
        """Measured L2 streaming-read GB/s, scattered 64-byte record fetches/s and 32-bit
        integer ops/s of this GPU (roofline denominators)."""
        p = hrr_peaks()
        self.check(hrr_measure_peaks(self.handle, C.byref(p)))
        return {"l2_read_gbs": p.l2_read_gbs, "record_fetches_per_s": p.record_fetches_per_s,
                "int_ops_per_s": p.int_ops_per_s}

    def last_cull_stats(self):
        v, a = _u64(), _u64()
        self.check(hrr_last_cull_stats(self.handle, C.byref(v), C.byref(a)))
        return int(v.value), int(a.value)

    def autotune(self, x, y, z, px, py, tree: "Tree", tau: float, pairs):
        """Fastest launch shape on these eyes: (tuning dict, median ms)."""
        E = hrr_eyes(_ptr(x), _ptr(y), _ptr(z), _ptr(px), _ptr(py))
        best = hrr_tuning()
        ms = C.c_double()
        self.check(hrr_autotune(self.handle, E, int(x.numel()), tree.handle, float(tau), _ptr(pairs),
                                int(pairs.shape[0]), C.byref(best), C.byref(ms)))
        return best.to_dict(), float(ms.value)

    def autotune_all(self, x, y, z, px, py, tree: "Tree", tau: float, pairs):
        """Every candidate tuning with its median time on these eyes: [(tuning dict, ms)]."""
        E = hrr_eyes(_ptr(x), _ptr(y), _ptr(z), _ptr(px), _ptr(py))
        need = _u32()
        hrr_autotune_all(self.handle, E, int(x.numel()), tree.handle, float(tau), _ptr(pairs),
                         int(pairs.shape[0]), None, None, 0, C.byref(need))
        n = int(need.value)
        tried = (hrr_tuning * n)()
        ms = (C.c_double * n)()
        got = _u32()
        self.check(hrr_autotune_all(self.handle, E, int(x.numel()), tree.handle, float(tau), _ptr(pairs),
                                    int(pairs.shape[0]), tried, ms, n, C.byref(got)))
        return [(tried[k].to_dict(), float(ms[k])) for k in range(int(got.value))]

    def range_min(self, a, b, r, out_min, out_argmin=None, variant: int = 0):
        self.check(hrr_range_min(self.handle, _ptr(a), _ptr(b), _ptr(r), _ptr(out_min),
                                 _ptr(out_argmin), int(a.numel()), variant))

    # -- accounting ------------------------------------------------------------------------
    def launch_count(self) -> int:
        n = _u64()
        self.check(hrr_launch_count(self.handle, C.byref(n)))
        return int(n.value)

    def set_timing(self, enable: bool):
        self.check(hrr_set_timing(self.handle, 1 if enable else 0))

    def kernel_time(self):
        ms, n = C.c_double(), _u64()
        self.check(hrr_kernel_time(self.handle, C.byref(ms), C.byref(n)))
        return float(ms.value), int(n.value)


class Batch:
    """Frames culled together in one persistent launch (optionally a recorded CUDA graph).

    ``frames`` is a list of dicts with keys: x, y, z, px, py (CUDA tensors of one frame's
    eyes), tree (Tree), tau, pairs (int32 tensor (cap, 2)); optional tile (uint32 tensor
    (h, w) or (d, h, w) on the device), sample_index, shift_offset, eye_visits (int32
    tensor)."""

    def __init__(self, ctx: "Context", frames, rangemin_variant: int = 0, use_graph: bool = True,
                 tuning=None):
        self.ctx = ctx
        self.n = len(frames)
        arr = (hrr_frame * self.n)()
        self._keep = frames  # the frames' tensors must outlive the batch
        for i, fr in enumerate(frames):
            tile = fr.get("tile")
            d, h, w = _tile_dims(tile)
            arr[i] = hrr_frame(
                hrr_eyes(_ptr(fr["x"]), _ptr(fr["y"]), _ptr(fr["z"]), _ptr(fr["px"]), _ptr(fr["py"])),
                int(fr["x"].numel()), fr["tree"].handle, _ptr(tile), w, h,
                float(fr["tau"]), int(fr.get("shift_offset", 0)),
                _ptr(fr["pairs"]) if fr["pairs"].shape[0] else None, int(fr["pairs"].shape[0]),
                _ptr(fr.get("eye_visits")), d, int(fr.get("sample_index", 0)))
        h = _P()
        tn = hrr_tuning.from_dict(tuning) or hrr_tuning(rangemin_variant, 0, 0, 0, 0)
        ctx.check(hrr_batch_create(ctx.handle, arr, self.n, C.byref(tn), 1 if use_graph else 0,
                                   C.byref(h)))
        self.handle = h

    def launch(self):
        self.ctx.check(hrr_batch_launch(self.ctx.handle, self.handle))

    def results(self):
        """(status, counts, visits): HRR_ERR_OVERFLOW is returned, not raised."""
        counts = (_u64 * self.n)()
        visits = (_u64 * self.n)()
        st = hrr_batch_results(self.ctx.handle, self.handle, counts, visits)
        if st not in (HRR_OK, HRR_ERR_OVERFLOW):
            self.ctx.check(st)
        return st, [int(c) for c in counts], [int(v) for v in visits]

    def destroy(self):
        if self.handle:
            self.ctx.check(hrr_batch_destroy(self.ctx.handle, self.handle))
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            if self.handle and self.ctx.handle:
                self.destroy()
        except Exception:
            pass


class Server:
    """Served culling with continuous batching (a scheduler thread inside the library).

    Jobs are eyes (CUDA tensors) against a resident Tree; submit() returns a ticket at once,
    wait()/poll() give the result, release() frees the job's output buffer."""

    def __init__(self, ctx: "Context", hbm_budget_bytes: int, slice_eyes: int = 0,
                 max_jobs: int = 1024, rangemin_variant: int = 0, tuning=None):
        self.ctx = ctx
        h = _P()
        tn = hrr_tuning.from_dict(tuning) or hrr_tuning(rangemin_variant, 0, 0, 0, 0)
        ctx.check(hrr_server_create(ctx.handle, int(hbm_budget_bytes), int(slice_eyes), int(max_jobs),
                                    C.byref(tn), C.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, x, y, z, px, py, tree: "Tree", tau: float, cap: int, tile=None,
               shift_offset: int = 0, sample_index: int = 0, refit=None) -> int:
        """Queue a job; ``refit`` = (x, y, z, intensity) device tensors of moved lights refits
        ``tree`` before the job's eyes (see hrr_job.refit)."""
        d, h, w = _tile_dims(tile)
        rl = hrr_lights(*(_ptr(a) for a in refit)) if refit is not None else hrr_lights()
        job = hrr_job(hrr_eyes(_ptr(x), _ptr(y), _ptr(z), _ptr(px), _ptr(py)), int(x.numel()),
                      tree.handle, _ptr(tile), w, h, float(tau), int(shift_offset), int(cap), d,
                      int(sample_index), rl)
        t = _u64()
        self.ctx.check(hrr_server_submit(self.handle, self.ctx.handle, C.byref(job), C.byref(t)))
        self._keep[int(t.value)] = (x, y, z, px, py, tile, refit)
        return int(t.value)

    @staticmethod
    def _res(r):
        return {"status": int(r.status), "count": int(r.count), "visits": int(r.visits),
                "dev_pairs": r.dev_pairs, "queue_s": float(r.queue_s), "latency_s": float(r.latency_s)}

    def poll(self, ticket: int):
        r = hrr_job_result()
        st = hrr_server_poll(self.handle, ticket, C.byref(r))
        if st not in (HRR_OK, HRR_PENDING):
            raise HRRError(st, "hrr_server_poll")
        return self._res(r)

    def wait(self, ticket: int, timeout_s: float = 600.0):
        r = hrr_job_result()
        st = hrr_server_wait(self.handle, ticket, float(timeout_s), C.byref(r))
        if st not in (HRR_OK, HRR_ERR_TIMEOUT):
            raise HRRError(st, "hrr_server_wait")
        out = self._res(r)
        out["wait_status"] = st
        return out

    def pairs(self, ticket: int, result) -> np.ndarray:
        """Copy a finished job's pairs to a host array of shape (n, 2), n <= count."""
        n = int(result["count"])
        out = np.empty((max(n, 1), 2), dtype=np.uint32)
        got = _u64()
        self.ctx.check(hrr_server_copy_pairs(self.handle, ticket, out.ctypes.data, n, C.byref(got)))
        return out[:int(got.value)]

    def release(self, ticket: int):
        self.ctx.check(hrr_server_release(self.handle, ticket))
        self._keep.pop(ticket, None)

    def stats(self):
        i = hrr_server_info()
        self.ctx.check(hrr_server_stats(self.handle, C.byref(i)))
        return {k: int(getattr(i, k)) for k, _ in hrr_server_info._fields_}

    def destroy(self):
        if self.handle:
            hrr_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):  # pragma: no cover
        try:
            self.destroy()
        except Exception:
            pass


class Scene:
    """A device-resident triangle hierarchy (occluders of the connections)."""

    def __init__(self, ctx: "Context", handle):
        self.ctx = ctx
        self.handle = handle

    def free(self):
        if self.handle:
            self.ctx.check(hrr_free_scene(self.ctx.handle, self.handle))
            self.handle = None


class Tree:
    """A device-resident light hierarchy owned by the library."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle
        n, h = _u32(), _u32()
        ctx.check(hrr_tree_info(handle, C.byref(n), C.byref(h), None))
        self.n_lights = int(n.value)
        self.height = int(h.value)

    def download(self):
        """(records as a NODE_DTYPE array, permutation) copied to host memory."""
        n = self.n_lights
        nodes = np.zeros(max(n - 1, 0), dtype=NODE_DTYPE)
        perm = np.zeros(n, dtype=np.uint32)
        self.ctx.check(hrr_tree_download(self.ctx.handle, self.handle,
                                         nodes.ctypes.data if n > 1 else None, perm.ctypes.data))
        return nodes, perm

    def free(self):
        if self.handle:
            self.ctx.check(hrr_free_light_tree(self.ctx.handle, self.handle))
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            if self.handle and self.ctx.handle:
                self.free()
        except Exception:
            pass
