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


class hrr_cull_opts(C.Structure):
    _fields_ = [("eye_visits", C.c_void_p), ("rangemin_variant", C.c_int),
                ("shift_offset", C.c_uint32)]


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
    "hrr_cull": (_i32, [_P, hrr_eyes, _u32, _P, _f32, _P, _u64, C.POINTER(_u64)]),
    "hrr_cull_ex": (_i32, [_P, hrr_eyes, _u32, _P, _f32, C.POINTER(hrr_cull_opts), _P, _u64,
                           C.POINTER(_u64)]),
    "hrr_last_cull_stats": (_i32, [_P, C.POINTER(_u64), C.POINTER(_u64)]),
    "hrr_range_min": (_i32, [_P, _P, _P, _P, _P, _P, _u64, _i32]),
    "hrr_build_light_tree_static": (_i32, [hrr_lights, _u32, _P, _P, C.POINTER(_u32), _P,
                                           C.c_char_p, C.c_size_t]),
}
STATIC_BUILD_MAX_LIGHTS = 65536
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


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
        tile = np.ascontiguousarray(tile, dtype=np.uint32)
        h, w = tile.shape
        self.check(hrr_set_shift_tile(self.handle, tile.ctypes.data, w, h))

    # -- hierarchy -------------------------------------------------------------------------
    def build_light_tree(self, x, y, z, intensity) -> "Tree":
        n = int(x.numel())
        L = hrr_lights(_ptr(x), _ptr(y), _ptr(z), _ptr(intensity))
        t = _P()
        self.check(hrr_build_light_tree(self.handle, L, n, C.byref(t)))
        return Tree(self, t)

    # -- culling ---------------------------------------------------------------------------
    def cull(self, x, y, z, px, py, tree: "Tree", tau: float, pairs, eye_visits=None,
             rangemin_variant: int = 0, shift_offset: int = 0):
        """Cull into ``pairs`` (uint32/int32 tensor of shape (cap, 2)); returns
        (status, count). HRR_ERR_OVERFLOW is returned, not raised."""
        n = int(x.numel())
        E = hrr_eyes(_ptr(x), _ptr(y), _ptr(z), _ptr(px), _ptr(py))
        cap = int(pairs.shape[0]) if pairs is not None else 0
        cnt = _u64()
        opts = hrr_cull_opts(_ptr(eye_visits), rangemin_variant, shift_offset)
        st = hrr_cull_ex(self.handle, E, n, tree.handle, float(tau), C.byref(opts),
                         _ptr(pairs) if cap else None, cap, C.byref(cnt))
        if st not in (HRR_OK, HRR_ERR_OVERFLOW):
            self.check(st)
        return st, int(cnt.value)

    def last_cull_stats(self):
        v, a = _u64(), _u64()
        self.check(hrr_last_cull_stats(self.handle, C.byref(v), C.byref(a)))
        return int(v.value), int(a.value)

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
