#!/usr/bin/env python
"""Benchmark of the hot path: fwd+bwd Mpixel/s of a training step (local render of K
subsets for V views, composition, L1 loss, backward, Adam) on seeded synthetic scenes.

Default workload: 10M Gaussians, SH degree 3, K = 8 k-d subsets, 16 views (8 x 1600x1064 and
8 x 1280x720) on a seeded orbit.  `value` is the batched path (one CUDA graph per step);
the plain per-view path is reported beside it.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpixel/s at 10M Gaussians, batched vs plain; serve p50/p99 ms"
UNIT = "Mpixel/s"

# Algorithmic FP32 work of the rasterisers per evaluated (pixel, list entry) pair, the unit
# the roofline counts: about 16 FP32-pipe instructions in the forward and 45 in the backward
# (plus one exp2 on the special-function unit, outside the FP32 peak).
OPS_PER_EVAL_FWD = 16
OPS_PER_EVAL_BWD = 45
# The bare arithmetic of the same events, reported beside it: an alpha evaluation (dx, dy,
# the conic's quadratic form, exp2, times opacity, clamp, threshold), a forward blend
# (1 - alpha, T update, stop test, alpha T, rgb and depth accumulation) and a backward
# contribution (T_i recovery 4, colour gradient 3, the dot product of dL/dC with the colour
# 3, dL/dalpha 2, opacity 1, dL/dpower 1, its five moments in dx, dy 7, the suffix term 1).
OPS_PER_ALPHA = 10
OPS_PER_BLEND = 8
OPS_PER_CONTRIB = 22
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_10m_k8")
    ap.add_argument("--n", type=int, default=0, help="override Gaussian count (profiling)")
    ap.add_argument("--views", type=int, default=0, help="override view count (profiling)")
    ap.add_argument("--tile", type=int, default=0,
                    help="tile side 8/16/32 (0: the autotuner picks tile and CTAs per SM)")
    ap.add_argument("--ctas-per-sm", type=int, default=0,
                    help="rasteriser CTAs per SM when --tile is given (0: one per work item)")
    ap.add_argument("--plain-steps", type=int, default=20)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--stale", action="store_true",
                    help="skip by each view's stale saturation state instead of the waves")
    ap.add_argument("--unfused-adam", action="store_true",
                    help="backward into gradient arrays and a separate Adam pass")
    ap.add_argument("--no-skip", action="store_true",
                    help="render every (view, subset, tile) item (no saturation skipping)")
    ap.add_argument("--whole-sort", action="store_true",
                    help="sort every tile segment whole (no selected prefixes of long ones)")
    ap.add_argument("--cpu-tile-fraction", type=float, default=1.0 / 48.0)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving run (0: skip it)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrivals per second")
    ap.add_argument("--serve-n", type=int, default=0, help="override the served scene's size")
    ap.add_argument("--city-steps", type=int, default=10,
                    help="timed steps of the 120M-Gaussian aerial-city training step (0: skip)")
    ap.add_argument("--city-warmup", type=int, default=3)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float) -> float:
    """Largest x over all ranks (the timing rule of the replica harness); x itself when
    there is no process group.  NCCL groups reduce on the GPU, gloo groups on the host."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(name, n_override=0, seed=3, rank=0, views_override=0):
    from paper_2606_18588_gb300 import inputs as I
    w = dict(I.WORKLOADS[name])
    n = n_override or w["n"]
    views = views_override or max(1, w["views"])
    sc, off, boxes, cams = I.cluster_case(n, seed, w["K"], views, w["sizes"], w["sh_degree"])
    if rank:
        cams = I.orbit_cameras(views, seed + 1 + 1000 * rank, w["sizes"])
    targets = [I.random_image(c.height, c.width, 100 + 17 * rank + i) for i, c in enumerate(cams)]
    desc = (f"{name}: {n} Gaussians SH{w['sh_degree']}, K={w['K']} k-d subsets (x/z), "
            f"{views} views " + "+".join(f"{sum(1 for c in cams if (c.width, c.height) == s)}x{s[0]}x{s[1]}"
                                         for s in w["sizes"]) + ", L1 loss vs seeded target, Adam")
    return sc, off, boxes, cams, targets, desc


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        mx = max((num(r[2]) for r in rows), default=float("nan"))
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        load = [s for s in sm if not math.isnan(s)]
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) for r in rows), default=None)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM traffic per unit of work measured by ncu (profiles/dram_traffic.json: per kernel its
# source file, that file's sha256 at the capture, bytes per unit and the unit).
KERNEL_SOURCE = {"raster_fwd": "raster.cu", "raster_bwd": "raster.cu", "project": "project.cu",
                 "fill": "bin.cu", "sort": "bin.cu", "project_bwd": "project_bwd.cu",
                 "composite": "composite.cu", "composite_bwd": "composite.cu"}


def measured_traffic(name, counts):
    """DRAM bytes per launch of `name` from the committed ncu table, scaled to this launch
    by its units of work; None if there is no entry or the kernel's source changed since
    the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)["kernels"]
    except (OSError, ValueError, KeyError):
        return None
    e = table.get(name)
    if not e:
        return None
    src = os.path.join(ROOT, "paper_2606_18588_gb300", "csrc", e["source"])
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if digest != e["sha256"]:
        return None
    units = counts.get(e["unit"])
    return None if units is None else float(e["bytes_per_unit"]) * units


def roofline(name, ms, counts, w, pk):
    """Roofline entry for kernel `name` of mean duration `ms` per launch."""
    V, N, K, nc, pixels = w["V"], w["N"], w["K"], w["nc"], w["pixels"]
    alu_peak = w["alu_peak"]  # T FP32 instr/s, derived from the device (device_peak)
    hbm = pk["hbm_gbs"]
    sec = ms / 1e3
    if name in ("raster_fwd", "raster_bwd"):
        if name == "raster_fwd":
            ev, more, per, unit = counts["alpha_fwd"], counts["blended"], OPS_PER_BLEND, OPS_PER_EVAL_FWD
        else:
            ev, more, per, unit = counts["alpha_bwd"], counts["contrib_bwd"], OPS_PER_CONTRIB, OPS_PER_EVAL_BWD
        a = ev * unit / sec / 1e12
        bare = (ev * OPS_PER_ALPHA + more * per) / sec / 1e12
        return {"kernel": name, "bound": "alu", "achieved": a, "peak": alu_peak,
                "unit": "T FP32 ops/s", "frac": a / alu_peak, "traffic": None,
                "work": f"{ev} evaluated (pixel, entry) pairs x {unit} FP32 instructions",
                "arithmetic": {"achieved": bare, "frac": bare / alu_peak,
                               "work": f"{ev} alpha evaluations x {OPS_PER_ALPHA} + {more} "
                                       f"{'blends' if name == 'raster_fwd' else 'contributions'}"
                                       f" x {per} FP32 ops"}}
    param_bytes = (3 + 3 + 4 + 1 + 3 * nc) * 4
    note = None
    # share of (view, subset, tile) work items inside the subsets' visible regions: the
    # composites read and write partial planes only there
    items = counts.get("items_total") or 0
    inside = 1.0 - (counts.get("outside_items", 0) / items) if items else 1.0
    if name == "sort":
        byts = counts["pairs"] * 16  # each tile segment read and written once
    elif name == "project":
        # parameters once, a tile count per (view, Gaussian), a record per kept one
        vis = counts.get("visible", V * N)
        byts = N * param_bytes + V * N * 4 + vis * 64
    elif name == "project_bwd":
        # tile counts of every (view, Gaussian); the 2-D gradients (48 B, read and cleared)
        # of the kept ones
        vis = counts.get("visible", V * N)
        if w.get("fused_adam"):
            # gradient from the views' 2-D gradients, then Adam in place: read p, m, v and
            # write p, m, v once
            byts = N * (6 * param_bytes) + V * N * 4 + vis * 96
            note = "Adam fused in: read p, m, v; write p, m, v; no gradient array"
        else:
            byts = N * (3 * param_bytes) + V * N * 4 + vis * 96
    elif name == "fill":
        vis = counts.get("visible", V * N)
        byts = V * N * 4 + vis * 32 + counts["pairs"] * 8
    elif name in ("composite", "composite_bwd"):
        per = 20 if name == "composite" else 36
        byts = pixels * (16 if name == "composite" else 12) + int(pixels * K * per * inside)
        note = (f"partial planes counted only inside the visible regions ({inside:.3f} of the "
                "work items)")
    elif name == "adam" and w.get("fused_adam"):
        byts = pixels * 3 * 12
        note = "the L1 loss alone (Adam runs inside project_bwd)"
    elif name == "adam":
        byts = N * param_bytes // 4 * 32 + pixels * 3 * 12
        note = "Adam over every parameter (read p, g, m, v; write p, m, v, g = 0) and the L1 loss"
    else:
        byts = V * N * 12
    a = byts / sec / 1e9
    out = {"kernel": name, "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
           "frac": a / hbm, "traffic": None, "work": f"{byts} algorithmic bytes"}
    if note:
        out["note"] = note
    return out


# ---------------------------------------------------------------- CPU oracle leg
def oracle_sample(sc, off, cam, frac, seed=0, reps=1, fixed_s=None):
    """Times the FP64 oracle's forward (local renders + composite) and backward on one view,
    restricted to a seeded fraction of its tiles, and once with no tiles (the fixed
    projection / binning cost; `fixed_s` reuses an earlier measurement of it).  Returns
    (extrapolated full-view seconds, info, threads, fixed seconds)."""
    import numpy as np
    from oracle import oracle as O
    o = O.opts()
    tw, th = (cam.width + 15) // 16, (cam.height + 15) // 16
    nt = tw * th
    rng = np.random.default_rng(seed)
    mask = np.zeros(nt, np.uint8)
    k = max(1, int(round(nt * frac)))
    mask[rng.choice(nt, k, replace=False)] = 1
    empty = np.zeros(nt, np.uint8)
    dl = rng.uniform(-1, 1, (3, cam.height, cam.width))

    def run(m):
        t = time.perf_counter()
        O.render_view(sc, off, cam, o, tile_mask=m)
        O.backward_view(sc, off, cam, dl, None, o, tile_mask=m)
        return time.perf_counter() - t
    t0 = fixed_s if fixed_s is not None else min(run(empty) for _ in range(reps))
    t1 = min(run(mask) for _ in range(reps))
    full = t0 + max(t1 - t0, 0.0) * nt / k
    info = (f"1 view {cam.width}x{cam.height}, all {len(off) - 1} subsets, forward+backward on "
            f"{k}/{nt} seeded tiles ({t1:.1f} s) plus the fixed projection/binning cost "
            f"({t0:.1f} s, no tiles), extrapolated to the full view")
    return full, info, O.num_threads(), t0


def cpu_baseline_small():
    """The oracle on the two small configurations (its fwd or fwd+bwd Mpixel/s on the host
    cores): the 10k-Gaussian plain forward at 256x256 (whole view, forward only) and the
    1M-Gaussian K = 4 1920x1080 forward + backward (a seeded 1/64 of the tiles plus the
    fixed projection cost, extrapolated to the full view)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2606_18588_gb300 import inputs as I
    out = {}
    sc, cam = I.plain_forward_case(0)
    t = time.perf_counter()
    O.render_view(sc, np.array([0, sc.n]), cam, O.opts())
    dt = time.perf_counter() - t
    out["plain_10k_sh0_256"] = {"value": cam.width * cam.height / dt / 1e6, "unit": UNIT,
                                "pass": "forward", "sample": "whole view", "seconds": dt}
    sc, off, _, cams = I.cluster_case(1_000_000, 2, 4, 1, [(1920, 1080)])
    full, info, _, _ = oracle_sample(sc, off, cams[0], 1.0 / 64.0)
    out["fwdbwd_1m_k4_1080p"] = {"value": cams[0].width * cams[0].height / full / 1e6,
                                 "unit": UNIT, "pass": "forward+backward", "sample": info}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    sc, off, _, cams, _, desc = make_workload(args.workload, args.n, views_override=args.views)
    cam = cams[0]
    times = []
    info = ""
    fixed = None  # the no-tile projection cost, measured once (steps differ in their tiles)
    for i in range(args.warmup + args.steps):
        full, info, cores, fixed = oracle_sample(sc, off, cam, args.cpu_tile_fraction, seed=i,
                                                 fixed_s=fixed)
        if i >= args.warmup:
            times.append(full)
    sec = statistics.mean(times)
    value = cam.width * cam.height / sec / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": info},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- serving
def serve_leg(args, ctx, rank, world):
    """Serving run: the serve_20m_k8 scene resident, a seeded Poisson stream of render
    requests (resolution uniform over 512^2, 1280x720, 1920x1080, 3840x2160; random
    poses around the scene) driven in real time through the native server."""
    import torch
    import torch.distributed as dist
    from paper_2606_18588_gb300 import inputs as I
    from paper_2606_18588_gb300 import serve
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import _subset_structs, scene_to_device
    w = I.WORKLOADS["serve_20m_k8"]
    n = args.serve_n or w["n"]
    t0 = time.perf_counter()
    sc, off, boxes, _ = I.cluster_case(n, 5 + rank, w["K"], 1, [(64, 64)], w["sh_degree"])
    gen_s = time.perf_counter() - t0
    from paper_2606_18588_gb300.visibility import front_to_back
    order_fn = None if args.no_skip else (lambda c: front_to_back(boxes, c.eye))
    dev = scene_to_device(sc)
    subs = _subset_structs(dev, off, sc.sh_degree)
    budget = 120 << 30
    srv = S.Server(ctx, subs, S.opts(), budget, slots=4, max_views=8)
    warm = serve.poisson_requests(8, 1e6, 999 + rank, (0, 0, 0), 25.0)
    serve.run(srv, warm, realtime=False, order_fn=order_fn)
    reqs = serve.poisson_requests(args.serve_requests, args.serve_rate, 7 + rank, (0, 0, 0), 25.0)
    if world > 1:
        dist.barrier()
    res = serve.run(srv, reqs, order_fn=order_fn)
    srv.close()
    out = res.summary()
    out.update({"workload": f"serve_20m_k8: {n} Gaussians SH{sc.sh_degree}, K={w['K']} resident, "
                            f"Poisson {args.serve_rate:g} req/s, resolutions uniform over "
                            "512x512/1280x720/1920x1080/3840x2160, random poses",
                "slots": 4, "max_views_per_launch": 8, "hbm_budget_gb": budget / 2**30,
                "saturation_skipping": order_fn is not None,
                "latency": "arrival (scheduled time) to the host seeing the result finished",
                "scene_gen_s": gen_s})
    del dev, subs
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- aerial city, 120M
def city_leg(args, rank, world, local, steps, warmup):
    """Training steps on the aerial-city scene (train_120m_k32): 120M Gaussians SH3 in K = 32
    k-d cells, each step a batch of 8 1920x1080 views sampled from a pool of 500 aerial
    cameras, forward + composite + L1 + backward + Adam over all parameters.  The scene is
    generated cell by cell straight into device memory; each step's views, subset orders
    and target images are set between graph replays (targets staged on the device first).
    Returns the measurements as a dict."""
    import torch
    import torch.distributed as dist
    from paper_2606_18588_gb300 import inputs as I
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import BatchedStep, _subset_structs, city_to_device
    from paper_2606_18588_gb300.visibility import orders_for_views

    w = I.WORKLOADS["train_120m_k32"]
    n, seed = args.n or w["n"], 4 + rank
    t0 = time.perf_counter()
    layout = I.city_layout(n, seed, w["K"], w["sh_degree"])
    pool = I.aerial_cameras(seed, size=w["sizes"][0])
    ctx = S.Context(local)
    dev = city_to_device(layout)
    gen_s = time.perf_counter() - t0
    nsteps = warmup + steps
    views = [[pool[i] for i in I.step_views(seed, s, len(pool), w["views"])] for s in range(nsteps)]
    orders = [None if args.no_skip else orders_for_views(layout.boxes, v) for v in views]
    px = sum(c.width * c.height for c in views[0])
    tgt = torch.empty((nsteps, 3 * px), device="cuda")
    for s, vs in enumerate(views):
        tgt[s].copy_(torch.cat([torch.from_numpy(I.random_image(c.height, c.width, 7919 * s + i))
                                .reshape(-1) for i, c in enumerate(vs)]))
    stream = torch.cuda.Stream()
    o = S.opts(tile=args.tile or 16)
    with torch.cuda.stream(stream):
        # pair capacity: the largest pair count over the steps' view sets (eager forwards of
        # a probe batch, whose memory the step's batch then reuses)
        pb = S.Batch(ctx, _subset_structs(dev, layout.offsets, layout.sh_degree), views[0], o,
                     0, stream=stream)
        rgb = torch.empty(pb.rgb_off[-1], device="cuda")
        need = 0
        for s in range(nsteps):
            pb.set_cameras(views[s], stream=stream)
            pb.set_order(orders[s])
            pb.forward(rgb, None, stream=stream)
            need = max(need, pb.status(stream)[1])
        ctx.device_status(stream)
        pb.close()
        del rgb
        cap = int(need * 1.05) + 1024
        st = BatchedStep(ctx, dev, layout.offsets, layout.sh_degree, views[0], None, o,
                         pair_capacity=cap, stream=stream, order=orders[0],
                         fused_adam=not args.unfused_adam)
        st.set_targets(tgt[0])
        st.batch.set_timing(True)
        if args.whole_sort:
            st.batch.set_prefix_sort(False)
        st.run()
        stream.synchronize()
        code, _ = st.status()
        if code != S.OK:
            raise RuntimeError(f"city step status {code}")
        counts = st.batch.counters(stream)  # the eager step's work
        launches0 = ctx.launch_count
        st.capture()
        launches_per_step = ctx.launch_count - launches0
        for s in range(warmup):
            st.set_views(views[s], orders[s])
            st.target.copy_(tgt[s], non_blocking=True)
            st.replay()
        stream.synchronize()
        clocks = Clocks(local)
        clocks.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(warmup, nsteps):
            st.set_views(views[s], orders[s])  # waits for the previous replay
            st.target.copy_(tgt[s], non_blocking=True)
            st.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clk = clocks.stop()
        code, _ = st.status()
        if code != S.OK:
            raise RuntimeError(f"city status after timed region {code}")
        ms = max_over_ranks(e0.elapsed_time(e1) / steps)
        kms = st.batch.kernel_times()  # the last timed replay's kernels
        st.close()
    ctx.close()
    del dev, tgt
    return {"metric": "fwd+bwd Mpixel/s (training step incl. Adam)",
            "value": px * world / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
            "steps": steps, "warmup": warmup,
            "workload": f"train_120m_k32: {n} Gaussians SH{layout.sh_degree} on an aerial city "
                        f"(1 km^2), K={layout.K} k-d subsets (x/z), {w['views']} views 1920x1080 "
                        f"per step sampled from {len(pool)} aerial cameras, L1 loss, Adam",
            "global_batch": w["views"] * world, "pixels_per_step": px * world, "tile": o.tile,
            "pair_capacity": cap, "saturation_skipping": not args.no_skip,
            "scene_gen_s": gen_s, "l2": "inputs larger than L2 (28 GB parameters)",
            "timing": "CUDA events around the timed steps; each step sets its views, orders "
                      "and targets between replays (a host wait for the previous replay)",
            "clocks": clk, "gpu_launches": launches_per_step * steps,
            "kernel_ms_last_step": kms, "counters_first_step": counts,
            # selected prefixes stay on only if the eager step handed back at most a quarter
            # of its prefix items (splx_batch_tune_prefix_sort, before the capture)
            "prefix_sort": (not args.whole_sort) and not (
                counts["prefix_items"] > 0 and 4 * counts["retried_items"] > counts["prefix_items"])}


def city_main(args):
    """`--workload train_120m_k32`: the aerial-city training step as the bench line."""
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    r = city_leg(args, rank, world, local, args.steps, args.warmup)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "global_batch", "pixels_per_step", "tile",
                                         "pair_capacity", "saturation_skipping", "scene_gen_s",
                                         "l2", "timing", "kernel_ms_last_step",
                                         "counters_first_step", "prefix_sort")},
            "roofline": None, "e2e": None, "clocks": r["clocks"],
            "gpu_launches": r["gpu_launches"]}
    line["config"]["parallelism"] = "replicas" if world > 1 else "single GPU"
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- our path
def timed_replays(st, steps, stream, barrier):
    """`steps` back-to-back replays of the step's graph with no host wait between them.
    Events recorded on the stream before each replay and after the last give the step
    times; the graph's timing ring gives every replay's per-kernel times, read after the
    loop.  Returns (total ms, per-step ms, per-replay kernel ms dicts)."""
    import torch
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    st.graph.set_timing_ring(steps)
    barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        evs[i].record(stream)
        st.replay()
    evs[steps].record(stream)
    torch.cuda.synchronize()
    barrier()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    total = evs[0].elapsed_time(evs[steps])
    ktimes = [st.batch.kernel_times(st.graph, i) for i in range(steps)]
    st.graph.set_timing_ring(0)
    return total, step_ms, ktimes


def batched_leg(args, ctx, dev, sc, off, cams, targets, o, ctas, order, stream, barrier, world):
    """Builds, captures and times the batched step (one CUDA graph per step).  Returns the
    step object (still open) and its measurements."""
    import torch
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import BatchedStep
    with torch.cuda.stream(stream):
        st = BatchedStep(ctx, dev, off, sc.sh_degree, cams, [torch.from_numpy(t) for t in targets],
                         o, stream=stream, order=order, fused_adam=not args.unfused_adam,
                         stale=args.stale and order is not None)
        st.batch.set_timing(True)
        st.batch.set_launch(ctas)
        if args.whole_sort:
            st.batch.set_prefix_sort(False)
        st.run()  # eager once: sizes everything, checks status
        stream.synchronize()
        code, pairs = st.status()
        if code != S.OK:
            raise RuntimeError(f"batched forward status {code}")
        counts = st.batch.counters(stream)
        counts["visible"] = st.batch.visible(stream)
        counts["items_total"] = (len(off) - 1) * sum(
            ((c.width + o.tile - 1) // o.tile) * ((c.height + o.tile - 1) // o.tile) for c in cams)
        launches0 = ctx.launch_count
        st.capture()
        launches_per_step = ctx.launch_count - launches0
        for _ in range(args.warmup):
            st.replay()
        stream.synchronize()
        code, _ = st.status()
        if code != S.OK:
            raise RuntimeError(f"status after warm-up {code}")
        total, step_ms, ktimes = timed_replays(st, args.steps, stream, barrier)
        code, _ = st.status()
        if code != S.OK:
            raise RuntimeError(f"status after timed region {code}")
    ms = max_over_ranks(total / args.steps)
    kmean = {k: statistics.mean(t[k] for t in ktimes) for k in ktimes[0]}
    kmean["loss+adam"] = max(ms - sum(kmean.values()), 0.0)
    return st, {"ms": ms, "step_ms_median": max_over_ranks(statistics.median(step_ms)),
                "value": st.pixels * world / (ms / 1e3) / 1e6, "kmean": kmean,
                "counts": counts, "launches_per_step": launches_per_step,
                "fused_adam": st.fused_adam}


def plain_leg(args, ctx, dev, sc, off, cams, targets, o, stream, barrier, world):
    """The plain per-view path (one render_partial per (view, subset), composite, loss and
    backward per view, one Adam), timed per step with CUDA events on its stream."""
    import torch
    from paper_2606_18588_gb300.train import PlainStep
    with torch.cuda.stream(stream):
        ps = PlainStep(ctx, dev, off, sc.sh_degree, cams, [torch.from_numpy(t) for t in targets],
                       o, stream=stream)
        for _ in range(max(1, min(args.warmup, 3))):
            ps.run()
        stream.synchronize()
        n = args.plain_steps
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
        barrier()
        torch.cuda.synchronize()
        for i in range(n):
            evs[i].record(stream)
            ps.run()
        evs[n].record(stream)
        torch.cuda.synchronize()
        barrier()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(n)]
    med = max_over_ranks(statistics.median(step_ms))
    mean = max_over_ranks(evs[0].elapsed_time(evs[n]) / n)
    px = ps.pixels * world
    del ps
    return {"mpixel_s": px / (med / 1e3) / 1e6, "ms_per_step_median": med,
            "ms_per_step_mean": mean, "steps": n, "timing": "CUDA events per step, median",
            "path": "one render_partial per (view, subset) + composite + L1 + backward per "
                    "view, one Adam; every subset rendered (no saturation skipping)"}


def device_peak(local):
    """FP32 peak derived from the device: SM count (CUDA device properties) x 128 FP32
    lanes x the maximum SM clock (nvidia-smi clocks.max.sm, else the measured-peaks file)."""
    import torch
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(local), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=20).stdout.strip()
        mhz = float(out.splitlines()[0])
    except Exception:
        pass
    src = "nvidia-smi clocks.max.sm"
    if not mhz:
        mhz = peaks()[0].get("sm_max_mhz", 2070.0)
        src = "MEASURED_PEAKS.json sm_max_mhz"
    return {"sms": sms, "fp32_lanes_per_sm": FP32_LANES_PER_SM, "sm_max_mhz": mhz,
            "tflops": sms * FP32_LANES_PER_SM * mhz * 1e6 / 1e12, "clock_source": src}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "train_120m_k32":
        return city_main(args)
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import scene_to_device

    def barrier():
        if world > 1:
            dist.barrier()

    sc, off, boxes, cams, targets, desc = make_workload(args.workload, args.n, rank=rank,
                                                        views_override=args.views)
    ctx = S.Context(local)
    dev = scene_to_device(sc)
    stream = torch.cuda.Stream()
    # saturation skipping: per view the front-to-back order of the k-d cells
    from paper_2606_18588_gb300.visibility import orders_for_views
    order = None if args.no_skip else orders_for_views(boxes, cams)
    tune = None
    if args.tile == 0:
        from paper_2606_18588_gb300.autotune import autotune
        tgt = torch.cat([torch.from_numpy(t).reshape(-1) for t in targets]).cuda()
        tune = autotune(ctx, dev, off, sc.sh_degree, cams, tgt, stream=stream, order=order)
        tile, ctas = tune.tile, tune.ctas_per_sm
        del tgt
    else:
        tile, ctas = args.tile, args.ctas_per_sm
    o = S.opts(tile=tile)
    dpk = device_peak(local)

    # ---- the headline: batched graph with saturation skipping (clocks sampled meanwhile)
    clocks = Clocks(local)
    clocks.start()
    st, head = batched_leg(args, ctx, dev, sc, off, cams, targets, o, ctas, order, stream,
                           barrier, world)
    clk = clocks.stop()
    ms, value, kmean, counts = head["ms"], head["value"], head["kmean"], head["counts"]
    pixels = st.pixels

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        with torch.cuda.stream(stream):
            host_t = torch.cat([torch.from_numpy(t).reshape(-1) for t in targets]).pin_memory()
            host_loss = torch.empty(1).pin_memory()
            # the public step with host targets: forward and update graphs, the target's
            # upload overlapping the forward on its own stream
            st.capture_split()
            for _ in range(args.warmup):
                st.step_from_host(host_t, host_loss)
            barrier()
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(args.steps):
                st.step_from_host(host_t, host_loss)
            t1.record(stream)
            torch.cuda.synchronize()
            barrier()
        ems = max_over_ranks(t0.elapsed_time(t1) / args.steps)
        e2e = {"value": pixels * world / (ems / 1e3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": host_t.numel() * 4, "d2h_bytes_per_step": 4,
               "path": "BatchedStep.step_from_host: pinned targets uploaded on a copy stream "
                       "while the forward graph runs, then the loss/backward/Adam graph and "
                       "the loss read back; no host wait between steps",
               "ms_per_step": ems}
    st.close()
    st = None

    # ---- like for like: the batched graph without saturation skipping, and the plain
    # per-view path, both rendering every subset
    noskip = None
    if not args.no_plain and order is not None:
        st0, h0 = batched_leg(args, ctx, dev, sc, off, cams, targets, o, ctas, None, stream,
                              barrier, world)
        st0.close()
        noskip = {"mpixel_s": h0["value"], "ms_per_step": h0["ms"],
                  "ms_per_step_median": h0["step_ms_median"], "steps": args.steps,
                  "kernel_ms": h0["kmean"], "timing": "CUDA events, graph replays back to back",
                  "path": "the batched graph with every subset rendered (no saturation skipping)"}
    # the same skipping driven by each view's state from its previous visit (the previous
    # step): one sort and one rasteriser launch per step instead of the waves
    stale = None
    if not args.no_plain and order is not None and not args.stale:
        import argparse
        st1, h1 = batched_leg(argparse.Namespace(**{**vars(args), "stale": True}), ctx, dev, sc,
                              off, cams, targets, o, ctas, order, stream, barrier, world)
        st1.close()
        stale = {"mpixel_s": h1["value"], "ms_per_step": h1["ms"],
                 "ms_per_step_median": h1["step_ms_median"], "steps": args.steps,
                 "kernel_ms": h1["kmean"], "timing": "CUDA events, graph replays back to back",
                 "path": "saturation skipping by the stale state of each view (set by the "
                         "previous step's composite), one launch per stage"}
    plain = None
    if not args.no_plain and args.plain_steps > 0:
        plain = plain_leg(args, ctx, dev, sc, off, cams, targets, o, stream, barrier, world)

    # ---- roofline of the dominant kernel
    pk, pk_src = peaks()
    wl = {"V": len(cams), "N": sc.n, "K": len(off) - 1, "nc": (sc.sh_degree + 1) ** 2,
          "pixels": pixels, "alu_peak": dpk["tflops"], "fused_adam": head["fused_adam"]}
    cand = {k: v for k, v in kmean.items() if k != "loss+adam"}
    dom = max(cand, key=cand.get)
    roof = roofline(dom, cand[dom], counts, wl, pk)
    roof["peak_source"] = (f"{pk_src} HBM copy (MEASURED_PEAKS.json)" if roof["bound"] == "hbm"
                           else "derived: SMs x 128 FP32 lanes x max SM clock, read from the device")
    roof["device"] = dpk
    roof["share_of_step"] = cand[dom] / ms
    roof["traffic"] = measured_traffic(dom, counts)
    # the other kernels whose algorithmic work the step's counters fix, against their roofs
    others = {}
    # with saturation skipping the sort and the forward rasteriser run as waves of view groups
    # on several streams side by side: only their span together is a kernel time, so the
    # forward's fraction is taken over that span (a lower bound) and the sort gets none
    overlapped = order is not None and len(cams) >= 2 and not args.stale
    for name in ("raster_fwd", "raster_bwd", "sort", "composite", "composite_bwd", "project",
                 "project_bwd", "fill", "adam"):
        t = kmean.get("loss+adam" if name == "adam" else name)
        if overlapped and name == "sort":
            continue
        if overlapped and name == "raster_fwd":
            t = kmean["raster_fwd"] + kmean["sort"]
        if t:
            r = roofline(name, t, counts, wl, pk)
            others[name] = {"bound": r["bound"], "achieved": r["achieved"], "unit": r["unit"],
                            "frac": r["frac"], "ms": t}
            if "arithmetic" in r:
                others[name]["frac_arithmetic"] = r["arithmetic"]["frac"]
            if "note" in r:
                others[name]["note"] = r["note"]
            if overlapped and name == "raster_fwd":
                others[name]["note"] = ("over the span of the waves (segment sorts and forward "
                                        "rasterisers of the view groups, overlapped): a lower "
                                        "bound")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "global_batch": len(cams) * world,
                       "pixels_per_step": pixels * world, "tile": tile,
                       "raster_ctas_per_sm": ctas,
                       "autotune": tune.as_dict() if tune else None,
                       "path": "batched: one CUDA graph per step (project + tile counts, scan, "
                               "fill tile buckets, per-tile depth sort, raster fwd, composite, L1 "
                               "loss, composite bwd, raster bwd, project bwd, Adam)",
                       "saturation_skipping": order is not None,
                       "prefix_sort": (not args.whole_sort) and not (
                           counts["prefix_items"] > 0
                           and 4 * counts["retried_items"] > counts["prefix_items"]),
                       "adam": ("fused into the projection adjoint (kernel_ms project_bwd)"
                                if head["fused_adam"] else "separate pass over the gradients"),
                       "waves": ("sort + raster_fwd of up to 4 view groups on their own "
                                 "streams, side by side; kernel_ms sort and raster_fwd are the "
                                 "first group's stream's intervals, their sum the waves' span")
                                if order is not None and not args.stale else None,
                       "stale_state": ("saturation skipping by each view's state from its "
                                       "previous visit (the previous step), one sort and one "
                                       "forward rasteriser launch per step"
                                       if args.stale and order is not None else None),
                       "timing": "CUDA events around the back-to-back graph replays (no host "
                                 "wait between them); per-kernel times from the graph's "
                                 "timing ring, every replay",
                       "ms_per_step_median": head["step_ms_median"],
                       "l2": "inputs larger than L2 (2.4 GB parameters, 10 GB projected records)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "batched_noskip": noskip, "batched_stale": stale, "plain": plain, "kernel_ms": kmean,
                       "counters": counts, "kernel_rooflines": others},
            "roofline": roof, "e2e": e2e, "clocks": clk,
            "gpu_launches": head["launches_per_step"] * args.steps}
    del dev
    torch.cuda.empty_cache()

    # ---- serving: resident 20M-Gaussian scene, Poisson requests of mixed resolution
    if args.serve_requests > 0:
        line["serve"] = serve_leg(args, ctx, rank, world)
    ctx.close()
    torch.cuda.empty_cache()

    # ---- the 120M-Gaussian aerial-city training step
    if args.city_steps > 0:
        line["train_120m_k32"] = city_leg(args, rank, world, local, args.city_steps,
                                          args.city_warmup)
        torch.cuda.empty_cache()

    # ---- CPU oracle baselines (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            full, info, cores, _ = oracle_sample(sc, off, cams[0], args.cpu_tile_fraction)
            line["cpu_baseline"] = {"value": cams[0].width * cams[0].height / full / 1e6,
                                    "unit": UNIT, "cores": cores, "kind": "oracle", "sample": info}
            line["cpu_baseline"]["other_configs"] = cpu_baseline_small()
        except Exception as ex:  # the baseline is reported, never required
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                                    "sample": f"failed: {ex}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
