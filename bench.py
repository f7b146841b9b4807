"""Benchmark of blue-noise dithered QMC hierarchical Russian roulette on one GB300.

One step is one pass of the whole culling path over one frame: build the light hierarchy
(Morton keys, radix sort, radix tree, refit) and cull every eye against it, on the
frame-sized workload (1920x1080 eyes on a heightfield, 2^20 Gaussian-mixture lights,
64x64 blue-noise shift tile, tau for ~64 accepted lights per eye). Inputs are resident in
HBM when timing starts; L2 is flushed between steps (a 512 MiB write outside the step's
events). The metric is effective pairs/s = N_e * N_l / step time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own frame (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "effective pairs/s (N_e*N_l/time) at 2M x 1M"
UNIT = "pairs/s"
L2_FLUSH_BYTES = 512 << 20
# measured peaks of this GPU type (written by the benchmark driver); fallbacks otherwise
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(args=None):
    """The frame workload; --eyes WxH / --lights N shrink it for profiler captures."""
    import synth
    width, height, n_lights = 1920, 1080, 1 << 20
    if args is not None:
        width, height = (int(v) for v in args.eyes.lower().split("x"))
        n_lights = args.lights
    return synth.scene_frame(width=width, height=height, n_lights=n_lights)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.rows = []
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"]
        except Exception:
            sel = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    import paper_1907_12343_gb300 as hrr

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    s = workload(args)
    n_e, n_l = len(s.eye_pos), len(s.light_pos)
    stream = torch.cuda.Stream(dev)
    ctx = hrr.Context(local, stream)
    ctx.set_shift_tile(s.tile)

    with torch.cuda.stream(stream):
        lp = torch.from_numpy(s.light_pos).to(dev)
        ep = torch.from_numpy(s.eye_pos).to(dev)
        L = [lp[:, k].contiguous() for k in range(3)] + [torch.from_numpy(s.intensity).to(dev)]
        E = [ep[:, k].contiguous() for k in range(3)]
        px = torch.from_numpy(s.px.view(np.int16)).to(dev)
        py = torch.from_numpy(s.py.view(np.int16)).to(dev)
        cap = int(n_e * 160)
        pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream.synchronize()
    tau = float(s.tau)

    form = {k: v for k, v in (("node_width", args.node_width), ("top_levels", args.top_levels)) if v} or None

    def step():
        tree = ctx.build_light_tree(*L, topology=TOPOLOGY)
        st, cnt = ctx.cull(*E, px, py, tree, tau, pairs, tuning=form)
        tree.free()
        if st != hrr.HRR_OK:
            raise RuntimeError(f"cull status {st}")
        return cnt, tree

    # warm-up
    for _ in range(args.warmup):
        cnt, _ = step()
    tree = ctx.build_light_tree(*L, topology=TOPOLOGY)
    height = tree.height
    tree.free()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ctx.set_timing(True)
    launches0 = ctx.launch_count()
    clocks.start()
    t0 = time.perf_counter()
    visits = []
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            ev[k][0].record(stream)
            cnt, _ = step()
            ev[k][1].record(stream)
            visits.append(ctx.last_cull_stats()[0])
            flush.fill_(k)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = ctx.launch_count() - launches0
    kern_ms, kern_n = ctx.kernel_time()
    ctx.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_rank = sum(step_ms) / len(step_ms) / 1e3
    value, t_step = aggregate_throughput(n_e * n_l, t_rank, dist, dev)

    # cull-only throughput and the traversal kernel's roofline figures
    cull_ms = kern_ms / max(kern_n, 1)
    V = statistics.median(visits)
    peaks, kind = _peaks()
    measured = ctx.measure_peaks()  # L2, record-fetch and integer denominators (untimed)
    roof = roofline(V, cnt, n_e, cull_ms, peaks, kind, clk, workload=f"{args.eyes}x{n_l}", n_l=n_l,
                    measured=measured, tile_bytes=int(np.asarray(s.tile).nbytes))
    if args.node_width == 4:
        # the algorithmic op count per visit is that of binary visits: not comparable
        roof.update(achieved=None, frac=None, ops_per_visit=None, node_width=4,
                    note="visits are nodes of width four; the op-based roofline is defined for binary visits")

    # end to end through the public API with host buffers
    e2e = None if args.no_e2e else run_e2e(ctx, s, dev, stream, args, cap)
    # the per-frame hierarchy update for moved lights, against a full build
    refit = run_refit(ctx, L, dev, stream) if ws == 1 else None
    # the step after the culling: weights and shadow segments of the accepted pairs
    connect = run_connect(ctx, E, L, tau, pairs, cnt, dev, stream) if ws == 1 else None
    rangemin = (run_rangemin(ctx, dev, stream, peaks, n=args.rangemin_queries)
                if ws == 1 and not args.no_rangemin else None)
    # several samples per light: psi(n) offsets and a space-time tile
    samples = run_samples(ctx, s, L, E, px, py, tau, pairs, stream) if ws == 1 else None
    del pairs, flush

    # the batched (64 uneven frames) and served (Poisson jobs) forms, 1 GPU only
    batched = served = None
    if ws == 1 and (args.batch_frames > 0):
        import synth
        frames = upload_frames(ctx, synth.batch_frames(args.batch_frames), dev)
        with torch.cuda.stream(stream):
            batched = run_batched(ctx, frames, stream, dev)
            if args.served_jobs > 0:
                import paper_1907_12343_gb300 as hrr_mod
                tn = {k: batched["tuning"][k] for k in hrr_mod.TUNING_FIELDS}
                # the GPU's job-by-job capacity on these frames (jobs/s); 200 jobs/s is several
                # times that, so the configuration's own rate only measures queueing
                cap_jobs = args.batch_frames / (batched["plain_job_by_job"]["ms"] / 1e3)
                served = {"capacity_jobs_per_s": cap_jobs,
                          "config": run_served(ctx, frames, stream, dev, args.served_jobs, 200.0, tuning=tn)}
                served["config"]["offered_load"] = 200.0 / cap_jobs
                # the same at a load the GPU can sustain: 70% of its job-by-job capacity, with
                # enough jobs that p99 is a tail and not the maximum
                served["sustainable"] = run_served(ctx, frames, stream, dev, args.sustained_jobs,
                                                   0.7 * cap_jobs, seed=12, tuning=tn)
                # and with each job refitting its frame's hierarchy to moved lights first
                served["sustainable_refit"] = run_served(ctx, frames, stream, dev, max(16, args.served_jobs // 2),
                                                         0.7 * cap_jobs, seed=13, tuning=tn,
                                                         refit_sets=moved_light_sets(frames, dev))
        for fr in frames:
            fr["tree"].free()

    result = None
    if rank == 0:
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32/f32", "data": "synthetic",
            "config": frame_config(args, n_e, n_l, tau, height, ws),
            "accepted_pairs": int(cnt), "accepted_per_eye": cnt / n_e, "node_visits": int(V),
            "cull_only": {"ms": cull_ms, "value": n_e * n_l / (cull_ms / 1e3), "unit": UNIT},
            "refit": refit,
            "connect": connect,
            "rangemin": rangemin,
            "samples": samples,
            "wall_s": wall,
            "roofline": roof,
            "e2e": e2e,
            "batched": batched,
            "served": served,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if ws == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(s, args.cpu_seconds)
        print(json.dumps(result), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return result


# Algorithmic work of one node visit on the frame workload with the cost-driven hierarchy
# (counted with the oracle's traversal over 3,000 evenly spaced eyes): 1.960 internal child
# tests x 19 ops (the box gap, 9; its square, 3 with fused multiply-adds; the distance floor
# and the scaled bound, 2; the value of the range minimum, 2; the division-free cull
# comparison, 3) + 0.973 new range minima x 51 integer ops + 0.988 inherited minima x 2 +
# 0.040 leaf tests x 17.
OPS_PER_VISIT = 1.960 * 19 + 0.973 * 51 + 0.988 * 2 + 0.040 * 17
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "cull_single_kernel_frame_1920x1080.md")
PROFILE_SMALL = os.path.join(ROOT, "profiles", "cull_single_kernel_frame_480x270.md")
TOPOLOGY = "cost"  # hierarchy shape of the benchmarked builds (set from --topology)
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1907_12343_gb300", "csrc", f)
                  for f in ("hrr_cull_kernel.cuh", "hrr_math.cuh")]


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments and with whitespace runs collapsed, so that a
    comment edit does not count as a change of the code (string literals in these sources
    hold no comment markers)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(files=None) -> str:
    """Hash of the code (comments and whitespace ignored) of the given sources, by default
    the traversal kernel's."""
    import hashlib
    h = hashlib.sha256()
    for f in files or KERNEL_SOURCES:
        with open(f, encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def build_source_hash() -> str:
    """The hierarchy build's source: the cull's traffic depends on the tree it walks."""
    return kernel_source_hash([os.path.join(ROOT, "paper_1907_12343_gb300", "csrc", "hrr_build.cu")])


def _profile_keys(path, topology=None):
    """The "- key: value" lines of a committed ncu summary, if it was taken on the current
    kernel and build sources and on this hierarchy shape (None otherwise)."""
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().split()[0] if v.strip() else ""
    if vals.get("kernel_source_sha256") != kernel_source_hash():
        return None
    if vals.get("topology") != (topology or TOPOLOGY):
        return None
    if vals.get("build_source_sha256") != build_source_hash():
        return None
    return vals


def profiled_traffic(workload="", topology=None):
    """DRAM bytes per cull launch from the committed ncu summary, if it was taken on the
    current kernel source, on this workload and on this hierarchy shape (null otherwise)."""
    vals = _profile_keys(PROFILE_SUMMARY, topology)
    if not vals or (workload and vals.get("workload_eyes") != workload):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def profiled_l2(topology=None):
    """L2 throughput of the cull kernel from the committed small-frame ncu summary (bytes/s
    through the L2 slices and their busy fraction), if taken on the current sources."""
    vals = _profile_keys(PROFILE_SMALL, topology)
    if not vals:
        return None
    try:
        return {"workload": vals["workload_eyes"], "l2_bytes_per_s": float(vals["l2_bytes_per_s"]),
                "l2_throughput_pct": float(vals["l2_throughput_pct"]),
                "l1_throughput_pct": float(vals["l1_throughput_pct"])}
    except (KeyError, ValueError):
        return None


def aggregate_throughput(units_per_rank: float, t_rank: float, dist=None, device="cpu"):
    """Whole-job throughput of a weak-scaled run: every rank processes units_per_rank in
    t_rank seconds; the job takes the slowest rank's time (the only collective of the
    benchmark, a max-reduction of one number). Returns (units/s over all ranks, max time)."""
    import torch
    ws = 1
    t = t_rank
    if dist is not None and dist.is_initialized():
        ws = dist.get_world_size()
        x = torch.tensor([t_rank], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return ws * units_per_rank / t, t


def roofline(V, accepted, n_e, cull_ms, peaks, kind, clk, workload="", n_l=0, measured=None, tile_bytes=0):
    """Roofline of the traversal kernel, which is bound by instruction issue: the node
    records (64 B per visit) stay in L2 and DRAM traffic is essentially the output.
    achieved = algorithmic ops per launch (node visits x OPS_PER_VISIT) / kernel time;
    peak = SMs x 4 schedulers x 32 lanes x maximum SM clock (one lane-op per lane per
    clock at full issue)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * 4 * 32 * mhz * 1e6
    sec = cull_ms / 1e3
    achieved = V * OPS_PER_VISIT / sec
    return {
        "bound": "alu",
        "achieved": achieved / 1e12,
        "peak": peak / 1e12,
        "unit": "Tops/s",
        "frac": achieved / peak,
        "traffic": profiled_traffic(workload),
        "peak_kind": f"derived from {sms} SMs x 128 lanes x {mhz:.0f} MHz ({kind} sm_max_mhz)",
        "kernel": "cull_single_kernel",
        "kernel_ms": cull_ms,
        "ops_per_visit": OPS_PER_VISIT,
        "node_visits_per_s": V / sec,
        "node_record_bytes_gbs": 64.0 * V / sec / 1e9,
        "fractions": other_fractions(V, accepted, n_e, n_l, sec, peaks, measured or {}, tile_bytes),
    }


def other_fractions(V, accepted, n_e, n_l, sec, peaks, measured, tile_bytes):
    """The traversal's other rooflines, against denominators measured on this GPU:
    - l2: node-record bytes (64 B per visit) against an L2 streaming read, and visits
      against scattered 64-byte record fetches (two 256-bit loads each, the same form);
    - hbm: the bytes that must cross HBM once (records 64 (N_l - 1), eyes 16 N_e, the tile,
      pairs 8 |A|) against the measured copy bandwidth;
    - int32: the algorithmic ops per visit against independent 32-bit op chains."""
    out = {}
    if measured.get("l2_read_gbs"):
        ach = 64.0 * V / sec / 1e9
        out["l2_stream"] = {"achieved_gbs": ach, "peak_gbs": measured["l2_read_gbs"],
                            "frac": ach / measured["l2_read_gbs"]}
    if measured.get("record_fetches_per_s"):
        out["record_fetch"] = {"achieved_per_s": V / sec, "peak_per_s": measured["record_fetches_per_s"],
                               "frac": V / sec / measured["record_fetches_per_s"]}
    if peaks.get("hbm_gbs"):
        unique = 64.0 * max(n_l - 1, 1) + 16.0 * n_e + tile_bytes + 8.0 * accepted
        out["hbm"] = {"unique_bytes": unique, "achieved_gbs": unique / sec / 1e9, "peak_gbs": peaks["hbm_gbs"],
                      "frac": unique / sec / 1e9 / peaks["hbm_gbs"]}
    l2 = profiled_l2()
    if l2 and measured.get("l2_read_gbs"):
        # the L2 traffic ncu counts on the small frame (every sector the L2 serves: records,
        # stack spills, output), against the measured L2 streaming read
        out["l2_ncu"] = dict(l2, frac_of_l2_stream=l2["l2_bytes_per_s"] / 1e9 / measured["l2_read_gbs"])
    if measured.get("int_ops_per_s"):
        ach = V * OPS_PER_VISIT / sec
        out["int32"] = {"achieved_per_s": ach, "peak_per_s": measured["int_ops_per_s"],
                        "frac": ach / measured["int_ops_per_s"]}
    return out


def run_e2e(ctx, s, dev, stream, args, cap):
    """Same metric through the C ABI with host buffers, every step: hrr_build_light_tree_host
    copies the lights from pinned host memory and builds the hierarchy, then hrr_cull_host
    reads the eyes from pinned host memory and writes the accepted pairs to pinned host
    memory (its slices' copies overlap the culling). Only the library moves data."""
    import numpy as np
    import torch
    import paper_1907_12343_gb300 as hrr

    n_e, n_l = len(s.eye_pos), len(s.light_pos)
    host_l = [torch.from_numpy(np.ascontiguousarray(s.light_pos[:, k])).pin_memory() for k in range(3)]
    host_l.append(torch.from_numpy(s.intensity).pin_memory())
    host_e = [torch.from_numpy(np.ascontiguousarray(s.eye_pos[:, k])).pin_memory() for k in range(3)]
    host_e += [torch.from_numpy(s.px.view(np.int16)).pin_memory(), torch.from_numpy(s.py.view(np.int16)).pin_memory()]
    host_pairs = torch.empty((cap, 2), dtype=torch.int32).pin_memory()
    h2d = sum(h.numel() * h.element_size() for h in host_l + host_e)
    steps = max(2, min(args.steps, 5))
    times, d2h = [], []
    with torch.cuda.stream(stream):
        for k in range(steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            tree = ctx.build_light_tree_host(*host_l, topology=TOPOLOGY)
            st, cnt = ctx.cull_host(*host_e, tree, float(s.tau), host_pairs)
            tree.free()
            if st != hrr.HRR_OK:
                raise RuntimeError(f"cull status {st}")
            stream.synchronize()
            dt = time.perf_counter() - t0
            if k > 0:  # first iteration warms the pinned buffers
                times.append(dt)
                d2h.append(cnt * 8 + 24)
    t = statistics.mean(times)
    return {"value": n_e * n_l / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(statistics.mean(d2h)), "ms_per_step": t * 1e3, "steps": steps}


# ---------------------------------------------------------------------------------------
# batched and served forms
# ---------------------------------------------------------------------------------------

def upload_frames(ctx, frames_np, dev):
    """Device copies of the batched workload's frames, each with a resident hierarchy and
    tile (the served form keeps exactly these resident across jobs)."""
    import numpy as np
    import torch
    out = []
    for s in frames_np:
        lp = torch.from_numpy(s.light_pos).to(dev)
        ep = torch.from_numpy(s.eye_pos).to(dev)
        L = [lp[:, k].contiguous() for k in range(3)] + [torch.from_numpy(s.intensity).to(dev)]
        tree = ctx.build_light_tree(*L, topology=TOPOLOGY)
        out.append({"lights": L, "x": ep[:, 0].contiguous(), "y": ep[:, 1].contiguous(), "z": ep[:, 2].contiguous(),
                    "px": torch.from_numpy(s.px.view(np.int16)).to(dev),
                    "py": torch.from_numpy(s.py.view(np.int16)).to(dev),
                    "tree": tree, "tau": float(s.tau), "tile_np": s.tile,
                    "tile": torch.from_numpy(np.ascontiguousarray(s.tile).view(np.int32)).to(dev),
                    "n_e": len(s.eye_pos), "n_l": len(s.light_pos)})
    torch.cuda.synchronize(dev)
    return out


def plain_frame(ctx, fr, pairs, stream, tuning=None):
    """One frame through hrr_cull on the context stream: (ms on the device, count)."""
    import torch
    import paper_1907_12343_gb300 as hrr
    ctx.set_shift_tile(fr["tile_np"])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    st, cnt = ctx.cull(fr["x"], fr["y"], fr["z"], fr["px"], fr["py"], fr["tree"], fr["tau"], pairs,
                       tuning=tuning)
    b.record(stream)
    b.synchronize()
    if st != hrr.HRR_OK:
        raise RuntimeError(f"plain cull status {st}")
    return a.elapsed_time(b), cnt


def run_batched(ctx, frames, stream, dev, runs=3):
    """All frames in one persistent launch replayed from a CUDA graph, against the same
    frames culled one hrr_cull call after another."""
    import torch
    import paper_1907_12343_gb300 as hrr
    total_pairs = sum(fr["n_e"] * fr["n_l"] for fr in frames)
    # One launch takes one tuning: that of the size class holding the most eyes, tuned on
    # a sample of its largest frame (the launch time follows the eye count).
    from paper_1907_12343_gb300.autotune import Autotuner, size_class
    by_class = {}
    for fr in frames:
        by_class.setdefault(size_class(fr["n_e"], fr["n_l"]), []).append(fr)
    cls, members = max(by_class.items(), key=lambda kv: sum(fr["n_e"] for fr in kv[1]))
    big = max(members, key=lambda fr: fr["n_e"])
    tuner = Autotuner(ctx)
    t_tune = time.perf_counter()
    ctx.set_shift_tile(big["tile_np"])
    entry = tuner.tune(big["x"], big["y"], big["z"], big["px"], big["py"], big["tree"], big["tau"],
                       n_lights=big["n_l"])
    t_tune = time.perf_counter() - t_tune
    tuning = Autotuner.launch_fields(entry)
    scratch = torch.empty((max(fr["n_e"] for fr in frames) * 200, 2), dtype=torch.int32, device=dev)
    plain_ms, counts = [], []
    for fr in frames:
        ms, cnt = plain_frame(ctx, fr, scratch, stream, tuning)
        plain_ms.append(ms)
        counts.append(cnt)
    del scratch
    for fr, cnt in zip(frames, counts):
        fr["count"] = cnt
        fr["pairs"] = torch.empty((cnt + 1024, 2), dtype=torch.int32, device=dev)
    b = hrr.Batch(ctx, frames, use_graph=True, tuning=tuning)
    b.launch()
    st, got, _ = b.results()
    if st != hrr.HRR_OK or got != counts:
        raise RuntimeError("batched counts differ from plain counts")
    times = []
    for _ in range(runs):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.launch()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        b.results()
    b.destroy()
    t_b = statistics.median(times) / 1e3
    t_p = sum(plain_ms) / 1e3
    return {"frames": len(frames), "eyes": sum(fr["n_e"] for fr in frames),
            "lights": sum(fr["n_l"] for fr in frames), "accepted_pairs": int(sum(counts)),
            "value": total_pairs / t_b, "unit": UNIT, "ms": t_b * 1e3, "graph": True,
            "plain_job_by_job": {"value": total_pairs / t_p, "ms": t_p * 1e3},
            "speedup_vs_plain": t_p / t_b,
            "tuning": dict(tuning, size_class=cls, sample_eyes=min(big["n_e"], tuner.sample),
                           sample_ms=entry["sample_ms"], tune_s=t_tune,
                           candidates=[dict(t, ms=round(ms, 3)) for t, ms in sorted(tuner.last_table,
                                                                                    key=lambda tm: tm[1])])}


def _latency_stats(lat):
    import numpy as np
    a = np.sort(np.asarray(lat))
    return {"p50_s": float(np.percentile(a, 50)), "p99_s": float(np.percentile(a, 99)),
            "max_s": float(a[-1])}


def run_connect(ctx, E, L, tau, pairs, n_pairs, dev, stream, n_tris=1 << 18, reps=3):
    """Connection evaluation of the frame's accepted pairs: Russian-roulette weights alone,
    and with shadow segments against n_tris seeded occluder triangles (about half the
    connections blocked). Median device times of hrr_connect; the scene build is timed
    once."""
    import torch
    import synth
    n_e = int(E[0].numel())
    tris = torch.from_numpy(synth.occluder_triangles(n_tris, 21, size=0.003)).to(dev)
    sums = torch.zeros(n_e, dtype=torch.float32, device=dev)
    vis = torch.zeros(max(int(n_pairs), 1), dtype=torch.uint8, device=dev)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), out

    with torch.cuda.stream(stream):
        scene_ms, scene = timed(lambda: ctx.build_scene(tris))
        t_plain, t_vis = [], []
        for k in range(reps + 1):
            ms, _ = timed(lambda: ctx.connect(*E, L, tau, pairs, n_pairs, eye_sum=sums))
            if k:
                t_plain.append(ms)
        for k in range(reps + 1):
            ms, _ = timed(lambda: ctx.connect(*E, L, tau, pairs, n_pairs, scene=scene, visible=vis, eye_sum=sums))
            if k:
                t_vis.append(ms)
        frac = float(vis[:n_pairs].float().mean().item()) if n_pairs else 0.0
        scene.free()
    m_plain, m_vis = statistics.median(t_plain), statistics.median(t_vis)
    return {"pairs": int(n_pairs), "weights_ms": m_plain, "weights_value": n_pairs / (m_plain / 1e3),
            "occluders": n_tris, "scene_build_ms": scene_ms, "visibility_ms": m_vis,
            "visibility_value": n_pairs / (m_vis / 1e3), "unit": "connections/s", "visible_fraction": frac}


def run_samples(ctx, s, L, E, px, py, tau, pairs, stream, n_samples=4):
    """Sec. 3's extra samples per light on the frame: sample n culls with the shift
    r_j + psi(n), psi(n) = n / golden ratio in 32-bit fixed point (a shift offset), and
    with layer n of a 64 x 64 x n_samples space-time tile. One cull per sample (device time
    from library-recorded events) and all samples in one traversal (hrr_cull_samples,
    CUDA events on the stream), with the accepted pairs of each sample."""
    import torch
    import synth
    tree = ctx.build_light_tree(*L, topology=TOPOLOGY)
    out = {"samples": n_samples}
    n_e = int(E[0].numel())
    fused_pairs = torch.empty((n_samples, 80 * n_e, 2), dtype=torch.int32, device=E[0].device)

    def fused(offsets, reps=3):
        ts, counts = [], None
        with torch_stream(stream):
            for k in range(reps + 1):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                st, counts, vis = ctx.cull_samples(*E, px, py, tree, tau, offsets, fused_pairs)
                b.record(stream)
                b.synchronize()
                if st != 0:
                    raise RuntimeError(f"cull_samples status {st}")
                if k:
                    ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        return {"ms": ms, "ms_per_sample": ms / len(offsets), "accepted_per_sample": counts,
                "sample_visits": vis[0], "records_fetched": vis[1],
                "value_per_sample": n_e * int(L[0].numel()) / (ms / len(offsets) / 1e3), "unit": UNIT}

    try:
        for form in ("psi_offset", "spacetime_tile"):
            if form == "spacetime_tile":
                ctx.set_shift_tile(synth.shift_tile_3d(64, 64, n_samples, 2))
            ms, acc = [], []
            for n in range(n_samples):
                kw = {"shift_offset": (n * 0x9E3779B9) & 0xFFFFFFFF} if form == "psi_offset" else {"sample_index": n}
                with torch_stream(stream):
                    ctx.set_timing(True)
                    st, cnt = ctx.cull(*E, px, py, tree, tau, pairs, **kw)
                    t, k = ctx.kernel_time()
                    ctx.set_timing(False)
                if st != 0:
                    raise RuntimeError(f"cull status {st}")
                ms.append(t / max(k, 1))
                acc.append(int(cnt))
            n_l = int(L[0].numel())
            out[form] = {"ms_per_sample": statistics.mean(ms), "accepted_per_sample": acc,
                         "value": n_e * n_l / (statistics.mean(ms) / 1e3), "unit": UNIT}
            offs = [(n * 0x9E3779B9) & 0xFFFFFFFF for n in range(n_samples)] if form == "psi_offset" else [0] * n_samples
            f = fused(offs)
            if f["accepted_per_sample"] != acc:
                raise RuntimeError(f"one-traversal samples disagree with per-sample culls: {f['accepted_per_sample']} {acc}")
            f["speedup_vs_per_sample_culls"] = statistics.mean(ms) * n_samples / f["ms"]
            out[form]["one_traversal"] = f
    finally:
        ctx.set_shift_tile(s.tile)
        tree.free()
        del fused_pairs
    return out


def torch_stream(stream):
    import torch
    return torch.cuda.stream(stream)


def run_rangemin(ctx, dev, stream, peaks, n=1 << 26, reps=5):
    """hrr_range_min over the 2^26 seeded log-uniform (a, b, r) queries of the range-minimum
    workload (1.34 GB of traffic, well above L2), inputs resident: median device time of reps
    launches, and its HBM roofline (20 B per query: a, b, r read, minimum and argmin
    written)."""
    import numpy as np
    import torch
    import synth
    a, b, r = synth.rangemin_queries(n, seed=3)
    ta, tb, tr = (torch.from_numpy(v.view(np.int32)).to(dev) for v in (a, b, r))
    vmin, karg = torch.empty_like(ta), torch.empty_like(ta)
    # a 512 MiB fill before each timed group flushes L2 and keeps the stream busy while the
    # launches are queued; four back-to-back launches per group (each longer than the
    # host's launch overhead), so the events time kernels, not launch latency
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    per_group = 4
    ts = []
    with torch.cuda.stream(stream):
        for k in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(k)
            e0.record(stream)
            for _ in range(per_group):
                ctx.range_min(ta, tb, tr, vmin, karg)
            e1.record(stream)
            e1.synchronize()
            if k >= 2:
                ts.append(e0.elapsed_time(e1) / per_group)
    ms = statistics.median(ts)
    gbs = 20.0 * n / (ms / 1e3) / 1e9
    hbm = float(peaks.get("hbm_gbs", 0.0)) or None
    return {"queries": n, "ms": ms, "queries_per_s": n / (ms / 1e3), "bytes_per_query": 20,
            "achieved_gbs": gbs, "hbm_peak_gbs": hbm, "frac": gbs / hbm if hbm else None}


def run_refit(ctx, L, dev, stream, reps=5):
    """Median device time of hrr_refit_light_tree (moved lights, same ids) and of a full
    hrr_build_light_tree over the frame's lights."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(17)
    moved = [torch.clamp(c + (torch.rand(c.shape, generator=gen, device=dev) - 0.5) * 0.04, 0.0, 1.0).contiguous()
             for c in L[:3]] + [L[3]]
    tree = ctx.build_light_tree(*L, topology=TOPOLOGY)
    t_refit, t_build = [], []
    with torch.cuda.stream(stream):
        for k in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.refit_light_tree(tree, *(moved if k % 2 == 0 else L))
            b.record(stream)
            b.synchronize()
            if k:
                t_refit.append(a.elapsed_time(b))
        for k in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            t2 = ctx.build_light_tree(*L, topology=TOPOLOGY)
            b.record(stream)
            b.synchronize()
            t2.free()
            if k:
                t_build.append(a.elapsed_time(b))
    tree.free()
    return {"n_lights": int(L[0].numel()), "refit_ms": statistics.median(t_refit),
            "build_ms": statistics.median(t_build)}


def moved_light_sets(frames, dev, seed=13, sets=2):
    """Per frame, `sets` device copies of its lights jittered in position (+-2% of the
    scene) and intensity (x U[0.5, 1.5]): the lights of later animation frames. Seeded
    torch generator on the device (timing input only; no result is compared)."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    out = []
    for fr in frames:
        x, y, z, inten = fr["lights"]
        per = []
        for _ in range(sets):
            moved = [torch.clamp(c + (torch.rand(c.shape, generator=gen, device=dev) - 0.5) * 0.04, 0.0, 1.0)
                     for c in (x, y, z)]
            moved.append(inten * (0.5 + torch.rand(inten.shape, generator=gen, device=dev)))
            per.append([m.contiguous() for m in moved])
        out.append(per)
    return out


def run_served(ctx, frames, stream, dev, n_jobs, rate, seed=11, budget=150 << 30, slice_eyes=1 << 20,
               tuning=None, refit_sets=None):
    """Poisson arrivals of frame-sized jobs against resident hierarchies and tiles, served
    with continuous batching, against the same arrival sequence processed job by job. With
    refit_sets, job k refits its frame's hierarchy to moved lights (set k mod 2) before its
    eyes, in both forms: the per-frame update before the hot path is part of the latency."""
    import threading as th
    import numpy as np
    import torch
    import synth
    import paper_1907_12343_gb300 as hrr
    gaps = -np.log(1.0 - synth.uniform01(seed, 50, n_jobs)) / rate
    arrive = np.cumsum(gaps) - gaps[0]
    which = np.minimum((synth.uniform01(seed, 51, n_jobs) * len(frames)).astype(int), len(frames) - 1)
    work = sum(frames[f]["n_e"] * frames[f]["n_l"] for f in which)
    moved = (lambda k: refit_sets[which[k]][k % 2]) if refit_sets is not None else (lambda k: None)
    # moved lights change the counts: reserve room and check counts only without them
    cap_of = (lambda fr: 2 * fr["count"] + 4096) if refit_sets is not None else (lambda fr: fr["count"] + 1024)

    # served
    srv = hrr.Server(ctx, budget, slice_eyes=slice_eyes, max_jobs=max(64, n_jobs), tuning=tuning)
    tickets = [None] * n_jobs
    t0 = time.perf_counter()

    def submitter():
        for k in range(n_jobs):
            dt = t0 + arrive[k] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            fr = frames[which[k]]
            tickets[k] = srv.submit(fr["x"], fr["y"], fr["z"], fr["px"], fr["py"], fr["tree"], fr["tau"],
                                    cap_of(fr), tile=fr["tile"], refit=moved(k))

    thr = th.Thread(target=submitter)
    thr.start()
    lat, mismatch = [], 0
    for k in range(n_jobs):
        while tickets[k] is None:
            time.sleep(0.0005)
        r = srv.wait(tickets[k], 3600.0)
        if r["status"] != hrr.HRR_OK or (refit_sets is None and r["count"] != frames[which[k]]["count"]):
            mismatch += 1
        lat.append(r["latency_s"])
        srv.release(tickets[k])
    thr.join()
    makespan = time.perf_counter() - t0
    stats = srv.stats()
    srv.destroy()

    # plain, job by job in arrival order on the same GPU
    scratch = torch.empty((max(cap_of(fr) for fr in frames), 2), dtype=torch.int32, device=dev)
    lat_p = []
    t0 = time.perf_counter()
    for k in range(n_jobs):
        dt = t0 + arrive[k] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        if refit_sets is not None:
            ctx.refit_light_tree(frames[which[k]]["tree"], *moved(k))
        plain_frame(ctx, frames[which[k]], scratch, stream, tuning)
        lat_p.append(time.perf_counter() - t0 - arrive[k])
    makespan_p = time.perf_counter() - t0
    return {"jobs": n_jobs, "rate_per_s": rate, "hbm_budget_gb": budget / 2**30, "slice_eyes": slice_eyes,
            "refit_per_job": refit_sets is not None,
            "value": work / makespan, "unit": UNIT, "latency": _latency_stats(lat),
            "max_active": stats["max_active"], "slices": stats["slices"], "mismatched_jobs": mismatch,
            "plain_job_by_job": {"value": work / makespan_p, "latency": _latency_stats(lat_p)}}


# ---------------------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------------------

def _oracle_sample(s, n_sample):
    import numpy as np
    n_e = len(s.eye_pos)
    ids = np.linspace(0, n_e - 1, num=n_sample).round().astype(np.uint32)
    return ids


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return name
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def cpu_baseline(s, target_seconds=15.0):
    """Oracle hierarchical culling on the host cores over an evenly spaced eye sample,
    scaled to a full frame: N_e N_l / (t_build + t_sample * N_e / n_sample); beside it the
    same on one core (a smaller sample), and the flat brute force (every pair) on the
    1024 x 4096 uniform workload."""
    import oracle
    import synth
    n_e, n_l = len(s.eye_pos), len(s.light_pos)
    t0 = time.perf_counter()
    tree = oracle.Tree(s.light_pos, s.intensity, topology=TOPOLOGY)
    t_build = time.perf_counter() - t0
    n = 512
    while True:
        ids = _oracle_sample(s, n)
        res = oracle.cull_hier(tree, s.eye_pos[ids], s.px[ids], s.py[ids], s.tile, s.tau, eye_ids=ids)
        if res["seconds"] * 2 >= target_seconds or n >= n_e:
            break
        n = min(n_e, int(n * max(2.0, target_seconds / max(res["seconds"], 1e-3))))
    t_full = t_build + res["seconds"] * n_e / n
    # one core: a sample of about a quarter of the time budget
    n1 = max(64, int(n * 0.25 * target_seconds / max(res["seconds"] * res["threads"], 1e-3)))
    ids1 = _oracle_sample(s, min(n1, n_e))
    r1 = oracle.cull_hier(tree, s.eye_pos[ids1], s.px[ids1], s.py[ids1], s.tile, s.tau, eye_ids=ids1, nthreads=1)
    t1_full = t_build + r1["seconds"] * n_e / len(ids1)
    # the flat brute force on the small uniform workload (4.2M pairs)
    u = synth.scene_uniform()
    tu = oracle.Tree(u.light_pos, u.intensity)
    fl = oracle.cull_flat(tu, u.eye_pos, u.px, u.py, u.tile, u.tau)
    pairs_u = len(u.eye_pos) * len(u.light_pos)
    return {"value": n_e * n_l / t_full, "unit": UNIT, "cores": res["threads"], "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"oracle tree build over all {n_l} lights ({t_build:.2f} s) + hierarchical "
                      f"culling of {n} evenly spaced eyes ({res['seconds']:.2f} s), scaled to "
                      f"{n_e} eyes",
            "one_core": {"value": n_e * n_l / t1_full, "unit": UNIT, "cores": r1["threads"],
                         "sample": f"{len(ids1)} evenly spaced eyes ({r1['seconds']:.2f} s) on one thread "
                                   f"+ the build, scaled to {n_e} eyes"},
            "flat_uniform_1024x4096": {"value": pairs_u / fl["seconds"], "unit": UNIT, "cores": fl["threads"],
                                       "seconds": fl["seconds"], "accepted_pairs": int(len(fl["pairs"]))}}


def frame_config(args, n_e, n_l, tau, height, ws):
    """The benchmark workload's description, the same for both arms."""
    return {"workload": f"frame {args.eyes} eyes x {n_l} Gaussian-mixture lights, "
                        "64x64 blue-noise tile, ~64 accepted/eye",
            "n_eyes": n_e, "n_lights": n_l, "tau": tau, "tree_height": height,
            "step": "build light tree + cull all eyes", "topology": TOPOLOGY,
            "l2": "flushed between steps (512 MiB write outside the step events)",
            "parallelism": f"replicas x{ws}"}


def run_reference(args):
    """The oracle as the reference arm: each step culls a bounded eye sample on the host."""
    import numpy as np
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    import oracle
    s = workload(args)
    n_e, n_l = len(s.eye_pos), len(s.light_pos)
    t0 = time.perf_counter()
    tree = oracle.Tree(s.light_pos, s.intensity, topology=TOPOLOGY)
    t_build = time.perf_counter() - t0
    n = args.ref_eyes
    ids = _oracle_sample(s, n)
    sub = (s.eye_pos[ids], s.px[ids], s.py[ids])
    for _ in range(args.warmup):
        oracle.cull_hier(tree, *sub, s.tile, s.tau, eye_ids=ids)
    times = []
    for _ in range(args.steps):
        res = oracle.cull_hier(tree, *sub, s.tile, s.tau, eye_ids=ids)
        times.append(res["seconds"])
    t = statistics.mean(times)
    value = n * n_l / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/f32",
            "data": "synthetic",
            "config": frame_config(args, n_e, n_l, float(s.tau), int(tree.height), ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["threads"], "kind": "oracle",
                             "sample": f"{n} evenly spaced eyes x all {n_l} lights per step "
                                       f"(hierarchical oracle; tree built once in {t_build:.2f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-eyes", type=int, default=2048)
    ap.add_argument("--eyes", default="1920x1080", help="frame size WxH (one eye per pixel)")
    ap.add_argument("--lights", type=int, default=1 << 20)
    ap.add_argument("--topology", choices=["cost", "radix"], default="cost",
                    help="hierarchy shape over the Morton order (the same accepted set)")
    ap.add_argument("--node-width", type=int, choices=[0, 2, 4], default=0,
                    help="traversal node width of the timed step (0: the library default)")
    ap.add_argument("--top-levels", type=int, choices=[0, 1, 6], default=0,
                    help="top levels the traversal evaluates from shared memory (1: none, 0: the library default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-rangemin", action="store_true", help="skip the 2^26-query range-minimum leg")
    ap.add_argument("--rangemin-queries", type=int, default=1 << 26, help="queries of the range-minimum leg")
    ap.add_argument("--batch-frames", type=int, default=64, help="0 skips the batched/served forms")
    ap.add_argument("--served-jobs", type=int, default=256,
                    help="jobs of the served run at the configuration's 200 jobs/s (0 skips the served form)")
    ap.add_argument("--sustained-jobs", type=int, default=2000,
                    help="jobs of the served run at 70%% of the GPU's job-by-job capacity")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)  # at least three untimed warm-up steps
    global TOPOLOGY
    TOPOLOGY = args.topology
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
