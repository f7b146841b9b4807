"""The allocation-free hierarchy build (hrr_build_light_tree_static) through the C ABI.

Some callers cannot call cudaMalloc (their device memory belongs to their own pool, or an
allocation could stall a real-time thread). For them the library builds a hierarchy into
caller-owned arrays using a fixed static working area. This test checks, on two calls in
a row (the second one smaller, so stale working memory from the first would show), that
the result is bit-identical to the allocating hrr_build_light_tree, that the second call
changes neither the device's free memory nor torch's reserved pool, and that light sets
above the fixed maximum are refused with a clear message.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import upload_scene

pytestmark = pytest.mark.gpu


def _static_build(hrr, g, n, memory=None):
    """One hrr_build_light_tree_static call into freshly allocated output arrays. With a
    list `memory`, appends the device's free bytes and torch's reserved bytes from just
    before and just after the call (outputs allocated before the first reading)."""
    import torch
    dev = torch.device("cuda:0")
    nodes = torch.zeros((max(n - 1, 1), 16), dtype=torch.int32, device=dev)
    perm = torch.zeros(n, dtype=torch.int32, device=dev)
    height = ctypes.c_uint32(12345)
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream(dev)
    L = hrr.hrr_lights(g["lx"].data_ptr(), g["ly"].data_ptr(), g["lz"].data_ptr(), g["li"].data_ptr())
    torch.cuda.synchronize(dev)
    before = (torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_reserved(dev))
    st = hrr.hrr_build_light_tree_static(L, n, nodes.data_ptr(), perm.data_ptr(), ctypes.byref(height),
                                         ctypes.c_void_p(stream.cuda_stream), err, 256)
    torch.cuda.synchronize(dev)
    after = (torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_reserved(dev))
    if memory is not None:
        memory.append((before, after))
    return st, nodes, perm, height.value, err.value.decode()


def _scene(n, seed):
    pos = synth.gaussian_mixture_lights(n, 16, seed=seed)
    inten = np.exp(synth.normal(seed, 3, n)).astype(np.float32)
    return {"light_pos": pos, "intensity": inten, "eye_pos": pos[:1],
            "px": np.zeros(1, np.uint16), "py": np.zeros(1, np.uint16)}


def test_static_build_equals_allocating_build_twice():
    import paper_1907_12343_gb300 as hrr
    ctx = hrr.Context(0)
    memory = []
    for n, seed in ((hrr.STATIC_BUILD_MAX_LIGHTS, 31), (3001, 32)):
        g = upload_scene(_scene(n, seed))
        tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"])
        ref_nodes, ref_perm = tree.download()
        st, nodes, perm, height, msg = _static_build(hrr, g, n, memory)
        assert st == hrr.HRR_OK, msg
        got_nodes = nodes.cpu().numpy().view(hrr.NODE_DTYPE).reshape(-1)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), ref_perm)
        assert got_nodes.tobytes() == ref_nodes.tobytes()
        assert height == tree.height
        tree.free()
    # Nothing is allocated: after the first call (which may load the library's GPU code on
    # this device), neither the device's free memory nor torch's pool changes across a call.
    (free0, res0), (free1, res1) = memory[1]
    assert free1 == free0, (free0, free1)
    assert res1 == res0, (res0, res1)
    ctx.close()


def test_static_build_refuses_oversized_light_sets():
    import paper_1907_12343_gb300 as hrr
    n = hrr.STATIC_BUILD_MAX_LIGHTS + 1
    g = upload_scene(_scene(n, 33))
    st, _, _, _, msg = _static_build(hrr, g, n)
    assert st == hrr.HRR_ERR_INVALID_ARG
    assert str(hrr.STATIC_BUILD_MAX_LIGHTS) in msg
