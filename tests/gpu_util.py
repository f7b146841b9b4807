"""Helpers shared by the GPU parity tests: upload seeded scenes and run the library."""
import numpy as np


def dev():
    import torch
    return torch.device("cuda:0")


def upload_scene(s):
    import torch
    d = dev()
    lp = torch.from_numpy(np.ascontiguousarray(s["light_pos"])).to(d)
    ep = torch.from_numpy(np.ascontiguousarray(s["eye_pos"])).to(d)
    out = {
        "lx": lp[:, 0].contiguous(), "ly": lp[:, 1].contiguous(), "lz": lp[:, 2].contiguous(),
        "li": torch.from_numpy(np.ascontiguousarray(s["intensity"])).to(d),
        "ex": ep[:, 0].contiguous(), "ey": ep[:, 1].contiguous(), "ez": ep[:, 2].contiguous(),
        "px": torch.from_numpy(np.ascontiguousarray(s["px"]).view(np.int16)).to(d),
        "py": torch.from_numpy(np.ascontiguousarray(s["py"]).view(np.int16)).to(d),
    }
    return out


def default_width() -> int:
    """Node width of the library's default traversal (per-eye visits count its nodes)."""
    import paper_1907_12343_gb300 as hrr
    return int(hrr.default_tuning()["node_width"])


def oracle_hier(tree, eye_pos, px, py, tile, tau, width=None, **kw):
    """The oracle's hierarchical traversal read with the given node width (default: the
    library's), so its per-eye visits compare with the GPU's."""
    import oracle
    return oracle.cull_hier(tree, eye_pos, px, py, tile, tau, width=width or default_width(), **kw)


def sorted_pairs(p):
    p = np.asarray(p, dtype=np.uint32).reshape(-1, 2)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def run_cull(ctx, g, tree, tau, cap=None, visits=False, variant=0, shift_offset=0, n_eyes=None, tuning=None):
    import torch
    n_e = g["ex"].numel() if n_eyes is None else n_eyes
    if cap is None:
        cap = max(1024, 256 * n_e)
    pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev())
    vis = torch.zeros(n_e, dtype=torch.int32, device=dev()) if visits else None
    st, cnt = ctx.cull(g["ex"][:n_e], g["ey"][:n_e], g["ez"][:n_e], g["px"][:n_e], g["py"][:n_e],
                       tree, tau, pairs, eye_visits=vis, rangemin_variant=variant,
                       shift_offset=shift_offset, tuning=tuning)
    out = pairs[:min(cnt, cap)].cpu().numpy().view(np.uint32)
    return st, cnt, out, (vis.cpu().numpy().view(np.uint32) if visits else None)
