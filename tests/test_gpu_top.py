"""The top slots the traversal's head reads, through the C ABI: after every build and every
refit, the 63 slots that follow a tree's binary records hold the top six levels of the
hierarchy in heap order (slot 0 the root; slots 2s + 1 and 2s + 2 the children of slot s),
each with its box, maximum intensity (a leaf: its position and intensity), leaf range, node
number and kind, bit-exact against a heap walk over the oracle's tree."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_util import upload_scene

pytestmark = pytest.mark.gpu

SLOTS = 63
EMPTY, INTERNAL, LEAF = 0, 1, 2
F = np.float32


@pytest.fixture(scope="module")
def ctx():
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    yield c
    c.close()


class _DeviceBytes:
    """A view of device memory that torch can wrap (the test only reads it)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3}


def _device_top(tree):
    """The top slots as a (63, 12) float32 array (three float4 per slot)."""
    import torch
    import paper_1907_12343_gb300 as hrr
    n, h, dev = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_void_p()
    assert hrr.hrr_tree_info(tree.handle, ctypes.byref(n), ctypes.byref(h), ctypes.byref(dev)) == 0
    base = dev.value + 64 * (n.value - 1)
    raw = torch.as_tensor(_DeviceBytes(base, SLOTS * 48), device="cuda").clone().cpu().numpy()
    return raw.view(np.float32).reshape(SLOTS, 12)


def _expected_top(t):
    """The same slots from the oracle's tree: a walk from the root along each slot's path."""
    out = np.zeros((SLOTS, 12), np.float32)
    u = out.view(np.uint32)
    for s in range(SLOTS):
        path = s + 1
        kind, first, last, node = INTERNAL, 0, t.n - 1, 0
        lo = hi = np.zeros(3, F)
        imax = F(0)
        for b in range(path.bit_length() - 2, -1, -1):
            if kind != INTERNAL:
                kind = EMPTY
                break
            sp = int(t.split[node])
            if (path >> b) & 1 == 0:
                last, node = sp, sp
            else:
                first, node = sp + 1, sp + 1
            if first == last:
                kind, lo, hi, imax = LEAF, t.pos[first], t.pos[first], t.inten[first]
            else:
                kind, lo, hi, imax = INTERNAL, t.lo[node], t.hi[node], t.imax[node]
        if kind == EMPTY:
            continue
        out[s, 0:3], out[s, 3], out[s, 4:7] = lo, imax, hi
        u[s, 7], u[s, 8], u[s, 9], u[s, 10] = first, last, node, kind
    return out


def _trees():
    rng = np.random.default_rng(29)
    cases = []
    for n in (2, 3, 40, 63, 64, 65, 3000):
        cases.append((f"uniform{n}", rng.random((n, 3)).astype(F), np.exp(rng.standard_normal(n)).astype(F), "radix"))
    x = (2.0 ** -np.arange(1, 22, dtype=np.float64)).astype(F)
    line = np.stack([x, np.full_like(x, 0.5), np.full_like(x, 0.5)], axis=1)
    lp = np.concatenate([line, (rng.random((600, 3)) * 1e-3).astype(F)]).astype(F)
    for topo in ("radix", "cost"):
        cases.append((f"line-{topo}", lp, np.ones(len(lp), F), topo))
    g = synth.gaussian_mixture_lights(50021, 16, seed=8)
    cases.append(("gaussian-cost", g, np.exp(synth.normal(8, 2, 50021)).astype(F), "cost"))
    return cases


@pytest.mark.parametrize("case", _trees(), ids=lambda c: c[0])
def test_top_slots_equal_the_oracle_after_build_and_refit(ctx, case):
    name, pos, inten, topo = case
    g = upload_scene({"light_pos": pos, "intensity": inten, "eye_pos": pos[:1], "px": np.zeros(1, np.uint16),
                      "py": np.zeros(1, np.uint16)})
    tree = ctx.build_light_tree(g["lx"], g["ly"], g["lz"], g["li"], topology=topo)
    t = oracle.Tree(pos, inten, topology=topo)
    got = _device_top(tree)
    assert got.tobytes() == _expected_top(t).tobytes(), name
    # moved lights, same ids: the refit rewrites the slots with the records
    rng = np.random.default_rng(len(pos))
    pos2 = (pos + rng.normal(scale=1e-3, size=pos.shape)).astype(F)
    inten2 = (inten * F(1.5)).astype(F)
    g2 = upload_scene({"light_pos": pos2, "intensity": inten2, "eye_pos": pos2[:1],
                       "px": np.zeros(1, np.uint16), "py": np.zeros(1, np.uint16)})
    ctx.refit_light_tree(tree, g2["lx"], g2["ly"], g2["lz"], g2["li"])
    t.refit(pos2, inten2)
    assert _device_top(tree).tobytes() == _expected_top(t).tobytes(), name
    tree.free()
