"""Host-side logic without a GPU: the autotuner's result cache, the serving request
generator and latency summary, and the replica harness's max-over-ranks timing on two
gloo ranks."""
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
