"""Host-side logic without a GPU: the autotuner's result cache, the serving request
generator and latency summary, the replica harness's max-over-ranks timing on two gloo
ranks, and the bench line's roofline accounting."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_autotune_cache_roundtrip(tmp_path):
    from paper_2606_18588_gb300 import autotune as A
    k1 = A.cache_key("GB300", 1000, 8, 3, [(1600, 1064), (1280, 720)])
    k2 = A.cache_key("GB300", 1000, 8, 3, [(1280, 720), (1600, 1064)])
    assert k1 == k2  # the view order does not matter
    assert A.cache_key("GB300", 1001, 8, 3, [(1280, 720)]) != A.cache_key("GB300", 1000, 8, 3, [(1280, 720)])
    path = str(tmp_path / "tune.json")
    assert A.load_cached(path, k1) is None
    r = A.TuneResult(16, 4, 12.5, [(8, 0, 14.0), (16, 4, 12.5)])
    A.store_cached(path, k1, r)
    A.store_cached(path, "other", A.TuneResult(8, 0, 1.0, []))
    got = A.load_cached(path, k1)
    assert (got.tile, got.ctas_per_sm, got.ms) == (16, 4, 12.5)
    assert got.table == [(8, 0, 14.0), (16, 4, 12.5)]
    with open(path, "w") as f:
        f.write("{not json")
    assert A.load_cached(path, k1) is None  # a damaged cache is a miss, not an error


def test_poisson_requests_and_summary():
    from paper_2606_18588_gb300 import serve
    reqs = serve.poisson_requests(4000, 200.0, 7, center=(0, 0, 0), radius=25.0)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1.0 / 200.0) < 0.05 / 200.0  # exponential gaps, mean 1/rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.06   # coefficient of variation 1
    sizes = {(r.cam.width, r.cam.height) for r in reqs}
    assert sizes == set(serve.RESOLUTIONS)
    for r in reqs[:50]:  # every camera looks at the centre: it projects to the image centre
        R, tc = np.asarray(r.cam.R, np.float64), np.asarray(r.cam.t, np.float64)
        p = R @ np.zeros(3) + tc
        assert p[2] > 0
        assert abs(r.cam.fx * p[0] / p[2]) < 1e-3 and abs(r.cam.fy * p[1] / p[2]) < 1e-3
    again = serve.poisson_requests(10, 200.0, 7, center=(0, 0, 0), radius=25.0)
    assert [r.arrival for r in again] == [r.arrival for r in reqs[:10]]  # seeded
    res = serve.ServeResult(4, 0, 2.0, np.array([1.0, 2.0, 3.0, 100.0]), 4_000_000)
    s = res.summary()
    assert s["req_per_s"] == 2.0 and s["mpixel_s"] == 2.0
    assert s["p50_ms"] == 2.5 and 3.0 < s["p99_ms"] <= 100.0


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.dist_env()[:2], bench.max_over_ranks(10.0 + 5.0 * rank)))
    finally:
        dist.destroy_process_group()


def test_replica_timing_is_max_over_two_gloo_ranks():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, (0, 2), 15.0), (1, (1, 2), 15.0)]
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5  # no process group: the value itself


def test_roofline_accounting_per_unit():
    # the bench line's roofline: rasterisers at 16 (forward) and 45 (backward) FP32
    # instructions per evaluated (pixel, entry) pair, their bare arithmetic beside it, and
    # HBM kernels by their algorithmic bytes per unit, each divided by the launch time
    sys.path.insert(0, ROOT)
    import bench
    counts = dict(alpha_fwd=4_000_000_000, blended=2_000_000_000, alpha_bwd=3_000_000_000,
                  contrib_bwd=1_500_000_000, pairs=400_000_000, visible=140_000_000,
                  items_total=1000, outside_items=600)
    w = dict(V=16, N=10_000_000, K=8, nc=16, pixels=21_000_000, alu_peak=40.0,
             fused_adam=True)
    pk = {"hbm_gbs": 6800.0}
    r = bench.roofline("raster_bwd", 20.0, counts, w, pk)
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(3e9 * 45 / 0.02 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 40.0)
    assert r["arithmetic"]["achieved"] == pytest.approx((3e9 * 10 + 1.5e9 * 22) / 0.02 / 1e12)
    r = bench.roofline("raster_fwd", 10.0, counts, w, pk)
    assert r["achieved"] == pytest.approx(4e9 * 16 / 0.01 / 1e12)
    assert r["arithmetic"]["achieved"] == pytest.approx((4e9 * 10 + 2e9 * 8) / 0.01 / 1e12)
    r = bench.roofline("sort", 5.0, counts, w, pk)
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(4e8 * 16 / 0.005 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
    # composites count the partial planes only inside the visible regions (40 % here)
    r = bench.roofline("composite", 1.0, counts, w, pk)
    assert r["achieved"] == pytest.approx((21e6 * 16 + int(21e6 * 8 * 20 * 0.4)) / 0.001 / 1e9)
    # the fused projection adjoint: read and write p, m, v once, plus the kept views' bytes
    r = bench.roofline("project_bwd", 2.0, counts, w, pk)
    param_bytes = (3 + 3 + 4 + 1 + 3 * 16) * 4
    assert r["achieved"] == pytest.approx((1e7 * 6 * param_bytes + 16e7 * 4 + 1.4e8 * 96)
                                          / 0.002 / 1e9)
