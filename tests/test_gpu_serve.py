"""Render server (continuous batching over several streams, HBM-budget admission): each
request's image is the same alone and in a mix of concurrent requests, equals the batched
forward, and matches the oracle; budget rejection and throughput statistics."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_18588_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [(200, 120), (96, 64), (131, 77), (256, 256), (64, 200), (17, 3)]


@pytest.fixture(scope="module")
def ctx():
    from paper_2606_18588_gb300 import splx as S
    c = S.Context()
    yield c
    c.close()


@pytest.fixture(scope="module")
def scene():
    sc, off, _, _ = I.cluster_case(30_000, 21, 4, 1, [(64, 64)])
    cams = [I.orbit_cameras(1, 100 + i, [SIZES[i % len(SIZES)]])[0] for i in range(12)]
    return sc, off, cams


def _subsets(dev, off, deg):
    from gpu_util import subset_struct
    return [subset_struct(dev, int(off[k]), int(off[k + 1]), deg) for k in range(len(off) - 1)]


def _serve(ctx, subs, cams, slots, max_views, budget=8 << 30, one_by_one=False, orders=None):
    from paper_2606_18588_gb300 import splx as S
    srv = S.Server(ctx, subs, S.opts(), budget, slots=slots, max_views=max_views)
    outs, status = {}, {}
    ids = []
    for i, c in enumerate(cams):
        out = torch.full((3, c.height, c.width), float("nan"), device="cuda")
        rid = srv.submit(c, out, None if orders is None else orders[i])
        outs[rid] = out
        ids.append(rid)
        while one_by_one and rid not in status:
            for r, st in srv.poll():
                status[r] = st
    while len(status) < len(cams):
        for r, st in srv.poll():
            status[r] = st
    torch.cuda.synchronize()
    assert srv.stats()["inflight"] == 0 and srv.stats()["queued"] == 0
    srv.close()
    return [outs[r] for r in ids], [status[r] for r in ids]


def test_results_same_alone_and_in_the_mix(ctx, scene):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import to_device
    sc, off, cams = scene
    dev = to_device(sc)
    subs = _subsets(dev, off, sc.sh_degree)
    alone, st_a = _serve(ctx, subs, cams, slots=1, max_views=1, one_by_one=True)
    mix, st_m = _serve(ctx, subs, cams, slots=3, max_views=4)
    assert all(s == S.OK for s in st_a + st_m)
    for a, m in zip(alone, mix):
        assert torch.equal(a, m)
        assert not torch.isnan(a).any()


def test_server_equals_batched_forward_and_oracle(ctx, scene):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import check_band, to_device
    sc, off, cams = scene
    dev = to_device(sc)
    subs = _subsets(dev, off, sc.sh_degree)
    got, st = _serve(ctx, subs, cams[:6], slots=2, max_views=3)
    assert all(s == S.OK for s in st)
    b = S.Batch(ctx, subs, cams[:6], S.opts())
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    torch.cuda.synchronize()
    for v in range(6):
        assert torch.equal(b.views(rgb)[v], got[v])
    b.close()
    ref = O.render_view(sc, off, cams[0], O.opts(), bounds=True)
    check_band(got[0].cpu().numpy(), ref["image"], ref["amb"], ref["flip"]["image"],
               label="served request 0")


def test_budget_admission_and_rejection(ctx, scene):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import to_device
    sc, off, cams = scene
    dev = to_device(sc)
    subs = _subsets(dev, off, sc.sh_degree)
    # a budget that fits about one small launch at a time: everything still finishes, in
    # several launches, with identical images
    ref, _ = _serve(ctx, subs, cams[:4], slots=1, max_views=1, one_by_one=True)
    small, st = _serve(ctx, subs, cams[:4], slots=4, max_views=4, budget=40 << 20)
    assert all(s == S.OK for s in st)
    for a, m in zip(ref, small):
        assert torch.equal(a, m)
    # a budget below one request's records fails it cleanly instead of faulting
    _, st = _serve(ctx, subs, cams[:2], slots=2, max_views=2, budget=1 << 20)
    assert all(s == S.ERR_BUDGET for s in st)


def test_poisson_driver_reports_latency(ctx, scene):
    from paper_2606_18588_gb300 import serve
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import to_device
    sc, off, _ = scene
    dev = to_device(sc)
    subs = _subsets(dev, off, sc.sh_degree)
    reqs = serve.poisson_requests(40, 400.0, 3, center=(0, 0, 0), radius=25.0,
                                  resolutions=((128, 128), (200, 120), (64, 64)))
    srv = S.Server(ctx, subs, S.opts(), 4 << 30, slots=3, max_views=4)
    res = serve.run(srv, reqs, keep={0, 5})
    srv.close()
    s = res.summary()
    assert s["requests"] == 40 and s["failed"] == 0
    assert 0 < s["p50_ms"] <= s["p99_ms"]
    assert set(res.outputs) == {0, 5}


def test_server_with_saturation_skipping(ctx):
    # per-request front-to-back orders: the same images as the batched forward with those
    # orders, alone and in a mix
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.visibility import orders_for_views
    from gpu_util import to_device
    sc, off, boxes, cams = I.cluster_case(120_000, 9, 8, 6, [(160, 120), (96, 64), (200, 150)])
    orders = orders_for_views(boxes, cams)
    dev = to_device(sc)
    subs = _subsets(dev, off, sc.sh_degree)
    alone, st_a = _serve(ctx, subs, cams, slots=1, max_views=1, one_by_one=True, orders=orders)
    mix, st_m = _serve(ctx, subs, cams, slots=3, max_views=4, orders=orders)
    assert all(s == S.OK for s in st_a + st_m)
    b = S.Batch(ctx, subs, cams, S.opts())
    b.set_order(orders)
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    torch.cuda.synchronize()
    for v in range(len(cams)):
        assert torch.equal(alone[v], mix[v])
        assert torch.equal(b.views(rgb)[v], alone[v])
    b.close()


def test_a_request_admitted_while_another_renders_overlaps_it_on_the_device(ctx):
    """Continuous batching: request B arrives after request A has been launched and while A
    is still on the GPU.  B is admitted into a free slot at once (two requests in flight on
    the host side), and on the device B's projection and tile counts finish before A's
    image is done, so the two launches' work overlaps (the server's per-request device
    timeline, splx_server_request_times)."""
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import to_device
    sc, off, _, _ = I.cluster_case(2_000_000, 12, 4, 1, [(64, 64)])
    dev = to_device(sc)
    subs = _subsets(dev, off, sc.sh_degree)
    cam_a = I.orbit_cameras(1, 40, [(3840, 2160)])[0]
    cam_b = I.orbit_cameras(1, 41, [(512, 512)])[0]
    srv = S.Server(ctx, subs, S.opts(), 32 << 30, slots=2, max_views=1)
    out_a = torch.empty(3, cam_a.height, cam_a.width, device="cuda")
    out_b = torch.empty(3, cam_b.height, cam_b.width, device="cuda")
    a = srv.submit(cam_a, out_a)
    done = dict(srv.poll())
    assert srv.stats()["inflight"] == 1 and srv.stats()["queued"] == 0  # A launched
    b = srv.submit(cam_b, out_b)
    done.update(srv.poll())
    st = srv.stats()
    assert a not in done and st["queued"] == 0 and st["inflight"] == 2  # B admitted beside A
    while len(done) < 2:
        done.update(srv.poll())
    assert done[a] == S.OK and done[b] == S.OK
    ta, tb = srv.request_times(a), srv.request_times(b)
    srv.close()
    assert ta["begin"] <= tb["begin"]
    assert tb["counted"] < ta["end"], (ta, tb)  # B's kernels ran while A was in flight
    # and each image equals its request served alone
    for cam, out in ((cam_a, out_a), (cam_b, out_b)):
        alone, st1 = _serve(ctx, subs, [cam], slots=1, max_views=1)
        assert st1 == [S.OK] and torch.equal(alone[0], out)


def test_serving_20m_poisson_stream_one_percent_checked_by_the_oracle(ctx):
    """The serving workload: 20M Gaussians SH3 resident in K = 8 k-d subsets, 2000 requests
    arriving as a seeded Poisson stream at 200 per second, resolutions uniform over 512^2,
    1280x720, 1920x1080 and 3840x2160, saturation skipping on (as the benchmark serves
    them).  A seeded 1 % of the requests (20) is checked against the oracle on 8 seeded
    tiles each: the oracle sees the Gaussians that a conservative host bound lets reach the
    sampled tiles, in their global order, which gives the full scene's pixels there.
    Pixels within 1e-4 outside the ambiguity band and within 1e-4 plus the flip bound
    inside it."""
    from city_util import reach_tiles, tile_sample
    from gpu_util import check_band, to_device
    from paper_2606_18588_gb300 import serve
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.visibility import front_to_back
    w = I.WORKLOADS["serve_20m_k8"]
    sc, off, boxes, _ = I.cluster_case(w["n"], 5, w["K"], 1, [(64, 64)], w["sh_degree"])
    dev = to_device(sc)
    subs = _subsets(dev, off, sc.sh_degree)
    reqs = serve.poisson_requests(2000, 200.0, 7, (0, 0, 0), 25.0)
    rng = np.random.default_rng(77)
    checked = sorted(rng.choice(len(reqs), size=len(reqs) // 100, replace=False).tolist())
    srv = S.Server(ctx, subs, S.opts(), 120 << 30, slots=4, max_views=8)
    order_fn = lambda c: front_to_back(boxes, c.eye)  # noqa: E731
    res = serve.run(srv, reqs, keep=set(checked), order_fn=order_fn)
    srv.close()
    assert res.failed == 0 and set(res.outputs) == set(checked)
    K = len(off) - 1
    for j, i in enumerate(checked):
        cam = reqs[i].cam
        mask, pix = tile_sample(cam, 8, 500 + i)
        idx, sub_off = [], [0]
        for k in range(K):
            part = sc.subset(int(off[k]), int(off[k + 1]))
            keep = np.nonzero(reach_tiles(part, cam, mask))[0] + int(off[k])
            idx.append(keep)
            sub_off.append(sub_off[-1] + keep.size)
        sub = sc.take(np.concatenate(idx))
        ref = O.render_view(sub, np.asarray(sub_off), cam, O.opts(), tile_mask=mask,
                            order=list(order_fn(cam)), bounds=True)
        got = res.outputs[i].cpu().numpy()
        check_band(got, ref["image"], ref["amb"], ref["flip"]["image"], where=pix,
                   budget=0.02, label=f"served request {i} ({cam.width}x{cam.height})")
        assert ref["T"][pix].min() < 0.5  # the sampled tiles see geometry
