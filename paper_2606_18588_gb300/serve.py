"""Serving loop: render requests of mixed resolution against a resident scene.

The scheduler itself is native (libsplx's splx_server_*): continuous batching over
several CUDA streams, admission by an HBM budget, launches that never block the host.
This module drives it with a request stream (arrival times in seconds, e.g. a seeded
Poisson process), records each request's latency from arrival to the host seeing it
finished, and summarises throughput and p50/p99 latency.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import splx as S
from .inputs import Camera, pinhole

RESOLUTIONS = ((512, 512), (1280, 720), (1920, 1080), (3840, 2160))


@dataclasses.dataclass
class Request:
    arrival: float  # seconds from the start of the run
    cam: Camera


def poisson_requests(n: int, rate: float, seed: int, center, radius: float,
                     resolutions=RESOLUTIONS, fov_deg: float = 60.0) -> list[Request]:
    """n requests with exponential inter-arrival times (rate per second), a resolution
    drawn uniformly from `resolutions` and a random pose on a sphere shell around
    `center` looking at it."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    center = np.asarray(center, np.float64)
    for i in range(n):
        w, h = resolutions[rng.integers(len(resolutions))]
        d = rng.standard_normal(3)
        d[1] = -abs(d[1]) * 0.5  # above the scene (y down)
        d /= np.linalg.norm(d)
        eye = center + d * radius * rng.uniform(0.8, 1.2)
        out.append(Request(float(t[i]), pinhole(w, h, fov_deg, eye, center)))
    return out


@dataclasses.dataclass
class ServeResult:
    n: int
    failed: int
    wall_s: float
    latencies_ms: np.ndarray
    pixels: int

    def summary(self) -> dict:
        lat = self.latencies_ms
        return {"requests": self.n, "failed": self.failed, "wall_s": self.wall_s,
                "req_per_s": self.n / self.wall_s if self.wall_s > 0 else None,
                "mpixel_s": self.pixels / self.wall_s / 1e6 if self.wall_s > 0 else None,
                "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "mean_ms": float(lat.mean()) if lat.size else None}


def run(server: S.Server, requests: list[Request], keep=None, realtime: bool = True,
        idle_sleep_s: float = 1e-4, order_fn=None) -> ServeResult:
    """Submits each request at its arrival time (realtime) or all at once, polls until all
    finished.  `keep` (a set of request indices) keeps those outputs: they are returned in
    the result's `outputs` attribute as {index: tensor}.  order_fn(camera), if given, gives
    each request's front-to-back subset order (saturation skipping)."""
    outs = {}
    id_to_idx = {}
    done_t = {}
    failed = 0
    i = 0
    n = len(requests)
    t0 = time.perf_counter()
    while len(done_t) < n:
        now = time.perf_counter() - t0
        while i < n and (not realtime or requests[i].arrival <= now):
            c = requests[i].cam
            out = torch.empty(3, c.height, c.width, device="cuda")
            rid = server.submit(c, out, None if order_fn is None else order_fn(c))
            id_to_idx[rid] = i
            if keep is not None and i in keep:
                outs[i] = out
            i += 1
        fin = server.poll()
        tnow = time.perf_counter() - t0
        for rid, st in fin:
            idx = id_to_idx[rid]
            done_t[idx] = tnow
            if st != S.OK:
                failed += 1
        if not fin:
            time.sleep(idle_sleep_s)
    wall = time.perf_counter() - t0
    arrivals = np.array([r.arrival if realtime else 0.0 for r in requests])
    lat = np.array([(done_t[j] - arrivals[j]) * 1e3 for j in range(n)])
    px = sum(r.cam.width * r.cam.height for r in requests)
    res = ServeResult(n, failed, wall, lat, px)
    res.outputs = outs
    return res
