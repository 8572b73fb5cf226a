"""Autotuner of the batched path's launch shape: tile side B in {8, 16, 32} x rasteriser
CTAs per SM (0 = one CTA per (view, subset, tile) work item, n > 0 = n persistent CTAs
per SM taking work items from a device counter).

Sec. 4.3 consolidates views so that every GPU stays busy; on one GB300 the same goal is a
launch shape that keeps the 152 SMs busy for the batch at hand, which depends on the
image sizes, the number of subsets and the Gaussians' screen sizes.  The tuner times the
differentiable part of a step (forward, L1 loss, backward; no optimiser update, so the
parameters are untouched) for every candidate with CUDA events and keeps the fastest.
The forward is bit-identical for every candidate (a pixel's blend does not depend on the
tile side); gradients differ only in the summation order of their atomics.
"""
from __future__ import annotations

import dataclasses
import statistics

import numpy as np
import torch

from . import splx as S
from .train import _subset_structs

TILES = (8, 16, 32)
CTAS_PER_SM = (0, 1, 2, 4, 8, 16)


@dataclasses.dataclass
class TuneResult:
    tile: int
    ctas_per_sm: int
    ms: float
    table: list  # (tile, ctas_per_sm, median ms) for every candidate that ran

    def as_dict(self):
        return {"tile": self.tile, "ctas_per_sm": self.ctas_per_sm, "ms": self.ms,
                "table": [list(r) for r in self.table]}


def _time(fn, stream, reps):
    fn()  # warm
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def autotune(ctx: S.Context, params: dict, offsets, sh_degree: int, cams, target: torch.Tensor,
             tiles=TILES, ctas=CTAS_PER_SM, reps: int = 3, stream=None,
             base_opts: S.Opts | None = None, order=None) -> TuneResult:
    """Times forward + L1 loss + backward of the V views x K subsets batch for every
    (tile, CTAs per SM) candidate.  `target` is the flat concatenated target image;
    `order` ([V, K] front-to-back subset orders) tunes the saturation-skipping forward."""
    stream = stream or torch.cuda.current_stream()
    offsets = np.asarray(offsets)
    subs = _subset_structs(params, offsets, sh_degree)
    grads = {k: torch.zeros_like(v) for k, v in params.items()}
    gsub = _subset_structs(grads, offsets, sh_degree, mutable=True)
    table = []
    with torch.cuda.stream(stream):
        for tile in tiles:
            o = S.opts(tile=tile) if base_opts is None else _with_tile(base_opts, tile)
            batch = S.Batch(ctx, subs, cams, o, 0, stream=stream)
            try:
                if order is not None:
                    batch.set_order(order)
                rgb = torch.empty(batch.rgb_off[-1], device="cuda")
                dL = torch.empty_like(rgb)
                loss = torch.zeros(1, device="cuda")
                fmax, bmax = batch.max_ctas_per_sm()
                cap = max(1, min(fmax, bmax))
                for c in ctas:
                    if c > cap:
                        continue
                    batch.set_launch(c)

                    def step():
                        batch.forward(rgb, None, stream=stream)
                        S.loss_l1(ctx, rgb, target, loss, dL, stream=stream)
                        batch.backward(dL, None, gsub, stream=stream)

                    ms = _time(step, stream, reps)
                    code, _ = batch.status(stream)
                    if code != S.OK:
                        raise RuntimeError(f"autotune tile {tile} ctas {c}: status {code}")
                    table.append((tile, c, ms))
            finally:
                batch.close()
    tile, c, ms = min(table, key=lambda r: r[2])
    del grads
    return TuneResult(tile, c, ms, table)


def _with_tile(o, tile):
    """Copy of a ctypes splx_opts with another tile side."""
    n = type(o)()
    for f, _ in o._fields_:
        setattr(n, f, getattr(o, f))
    n.tile = tile
    return n


# ---------------------------------------------------------------- result cache
def cache_key(gpu_name: str, n: int, K: int, sh_degree: int, sizes) -> str:
    """Key of a tuning result: the GPU model and the batch's shape (Gaussian count, subsets,
    SH degree, the multiset of view resolutions)."""
    res = ",".join(f"{w}x{h}" for w, h in sorted((int(w), int(h)) for w, h in sizes))
    return f"{gpu_name}|n={int(n)}|K={int(K)}|deg={int(sh_degree)}|{res}"


def load_cached(path: str, key: str) -> TuneResult | None:
    import json
    import os
    if not path or not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            d = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not d:
        return None
    return TuneResult(int(d["tile"]), int(d["ctas_per_sm"]), float(d["ms"]),
                      [tuple(r) for r in d.get("table", [])])


def store_cached(path: str, key: str, r: TuneResult) -> None:
    import json
    import os
    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
    data[key] = r.as_dict()
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1)
    os.replace(tmp, path)


def autotune_cached(ctx: S.Context, params: dict, offsets, sh_degree: int, cams,
                    target: torch.Tensor, cache_path: str | None = None, **kw) -> TuneResult:
    """autotune() with its result kept in a JSON file per (GPU model, batch shape)."""
    n = int(params["means"].shape[0])
    key = cache_key(torch.cuda.get_device_name(), n, len(offsets) - 1, sh_degree,
                    [(c.width, c.height) for c in cams])
    if cache_path:
        hit = load_cached(cache_path, key)
        if hit is not None:
            return hit
    r = autotune(ctx, params, offsets, sh_degree, cams, target, **kw)
    if cache_path:
        store_cached(cache_path, key, r)
    return r
