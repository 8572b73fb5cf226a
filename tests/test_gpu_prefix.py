"""Selected-prefix sort of long tile segments (batches): results equal those of whole
segment sorts, bit for bit for images and transmittances and within the atomics' rounding
for gradients, on scenes that reach each of its routes: a prefix that every pixel
saturates within, a prefix at whose end pixels are still blending (the item is rendered
again after a whole sort), and a segment with no prefix at all (every key in the nearest
depth bin).  With and without saturation-skipping waves, and against the plain per-view
path."""
import numpy as np
import pytest

from paper_2606_18588_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def ctx():
    from paper_2606_18588_gb300 import splx as S
    c = S.Context()
    yield c
    c.close()


def _split(sc, K):
    perm, off, boxes = I.kd_partition(sc.means, K)
    return sc.take(perm), off, boxes


def _dense():
    # 40k Gaussians of half opacity over a 64 x 64 view: ~3000 keys per tile, pixels
    # saturate inside their nearest 2048
    sc = I.uniform_scene(40_000, 71, 1, log_scale_mu=-3.0)
    return _split(sc, 2)


def _faint():
    # faint Gaussians: pixels of long segments still blend after 2048 entries
    sc = I.uniform_scene(40_000, 72, 1, log_scale_mu=-3.5)
    sc.opacity_logits[:] = sc.opacity_logits - 2.5
    return _split(sc, 2)


def _planar():
    # 6000 Gaussians on the plane z = 0 facing the camera: every key of a tile has the same
    # depth bits, so no prefix below a depth threshold exists
    sc = I.uniform_scene(6_000, 73, 0, log_scale_mu=-3.2, extent=0.25)
    sc.means[:, 2] = 0.0
    return _split(sc, 2)


def _cams():
    return [I.pinhole(64, 64, 60.0, (0.0, 0.0, -3.0), (0, 0, 0)),
            I.pinhole(80, 48, 50.0, (0.2, -0.1, -3.2), (0, 0, 0))]


def _run(ctx, sc, off, cams, order, prefix, dL=None, tile=16):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import params_struct, subset_struct, to_device, zeros_like_params
    dev = to_device(sc)
    K = len(off) - 1
    subs = [subset_struct(dev, int(off[k]), int(off[k + 1]), sc.sh_degree) for k in range(K)]
    b = S.Batch(ctx, subs, cams, S.opts(tile=tile))
    b.set_prefix_sort(prefix)
    if order is not None:
        b.set_order(order)
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    T = torch.empty(b.total_pixels, device="cuda")
    b.forward(rgb, T)
    g = None
    if dL is not None:
        g = zeros_like_params(dev)
        b.backward(dL, None, [params_struct(g, int(off[k]), int(off[k + 1]), sc.sh_degree)
                              for k in range(K)])
    torch.cuda.synchronize()
    code, pairs = b.status()
    assert code == S.OK and pairs > 0
    counts = b.counters()
    out = (rgb.clone(), T.clone(), g, counts, [v.clone() for v in b.views(rgb)])
    b.close()
    return out


@pytest.mark.parametrize("make,route", [(_dense, "prefix"), (_faint, "retry"),
                                        (_planar, "none")])
@pytest.mark.parametrize("waves", [False, True])
def test_prefix_sort_equals_whole_sort(ctx, make, route, waves):
    from gpu_util import rel_l2
    from paper_2606_18588_gb300.visibility import orders_for_views
    sc, off, boxes = make()
    cams = _cams()
    order = orders_for_views(boxes, cams) if waves else None
    npix = sum(3 * c.width * c.height for c in cams)
    rng = np.random.default_rng(5)
    dL = torch.from_numpy(rng.standard_normal(npix).astype(np.float32)).cuda()
    rgb1, T1, g1, c1, _ = _run(ctx, sc, off, cams, order, True, dL)
    rgb0, T0, g0, c0, _ = _run(ctx, sc, off, cams, order, False, dL)
    assert c0["prefix_items"] == 0 and c0["retried_items"] == 0
    if route == "none":
        assert c1["retried_items"] > 0  # handed on without a prefix
    else:
        assert c1["prefix_items"] > 0
        if route == "retry":
            assert c1["retried_items"] > 0
        else:
            assert c1["retried_items"] < c1["prefix_items"]
    assert torch.equal(rgb1, rgb0)
    assert torch.equal(T1, T0)
    for k in GROUPS:
        assert rel_l2(g1[k].cpu().numpy(), g0[k].cpu().numpy()) < 1e-5, k


@pytest.mark.parametrize("tile", [8, 32])
def test_prefix_sort_at_other_tile_sizes(ctx, tile):
    # the rasterisers' other launch shapes on the prefix and hand-back routes, with waves
    from paper_2606_18588_gb300.visibility import orders_for_views
    for make in (_dense, _faint):
        sc, off, boxes = make()
        cams = _cams()
        order = orders_for_views(boxes, cams)
        rgb1, T1, _, c1, _ = _run(ctx, sc, off, cams, order, True, tile=tile)
        rgb0, T0, _, _, _ = _run(ctx, sc, off, cams, order, False, tile=tile)
        assert c1["prefix_items"] + c1["retried_items"] > 0, (make.__name__, tile)
        assert torch.equal(rgb1, rgb0) and torch.equal(T1, T0), (make.__name__, tile)


def test_prefix_sort_equals_plain_path(ctx):
    # without waves the batch renders every subset like the per-view path: bit for bit
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import render_view, to_device
    for make in (_dense, _faint, _planar):
        sc, off, _ = make()
        cams = _cams()
        _, _, _, counts, views = _run(ctx, sc, off, cams, None, True)
        assert counts["prefix_items"] + counts["retried_items"] > 0
        dev = to_device(sc)
        for v, cam in enumerate(cams):
            img, _, _, states = render_view(ctx, dev, off, cam, S.opts(), sc.sh_degree)
            for st in states:
                st.close()
            assert torch.equal(views[v], img), (make.__name__, v)


def test_prefix_sort_in_a_captured_graph(ctx):
    # the retry route's launches inside a graph: replays equal the eager forward
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    sc, off, _ = _faint()
    cams = _cams()
    dev = to_device(sc)
    subs = [subset_struct(dev, int(off[k]), int(off[k + 1]), sc.sh_degree)
            for k in range(len(off) - 1)]
    b = S.Batch(ctx, subs, cams, S.opts())
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    torch.cuda.synchronize()
    assert b.counters()["retried_items"] > 0
    ref = rgb.clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        S.graph_begin(ctx, s)
        b.forward(rgb, stream=s)
        gr = S.graph_end(ctx, s)
        for _ in range(2):
            rgb.zero_()
            gr.launch(s)
    s.synchronize()
    assert torch.equal(rgb, ref)
    gr.close()
    b.close()


def test_prefix_sort_switch_needs_a_batch_state(ctx):
    from paper_2606_18588_gb300 import splx as S
    sc, off, _ = _dense()
    cams = _cams()[:1]
    from gpu_util import subset_struct, to_device
    dev = to_device(sc)
    b = S.Batch(ctx, [subset_struct(dev, int(off[k]), int(off[k + 1]), sc.sh_degree)
                      for k in range(len(off) - 1)], cams, S.opts())
    b.set_prefix_sort(False)
    b.set_prefix_sort(True)
    b.close()


@pytest.mark.parametrize("make", [_dense, _faint, _planar])
def test_prefix_sort_tuning_follows_the_hand_back_share(ctx, make):
    # splx_batch_tune_prefix_sort keeps the selected prefixes only if at most a quarter of
    # the last eager forward's prefix items went back to the whole sort; the images stay
    # those of whole sorts either way
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    sc, off, _ = make()
    cams = _cams()
    dev = to_device(sc)
    b = S.Batch(ctx, [subset_struct(dev, int(off[k]), int(off[k + 1]), sc.sh_degree)
                      for k in range(len(off) - 1)], cams, S.opts())
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    c1 = b.counters()
    ref = rgb.clone()
    b.tune_prefix_sort()
    keep = not (c1["prefix_items"] > 0 and 4 * c1["retried_items"] > c1["prefix_items"])
    if make is _faint:
        assert not keep  # long lists of faint Gaussians: most prefixes are handed back
    b.forward(rgb)
    torch.cuda.synchronize()
    c2 = b.counters()
    assert (c2["prefix_items"] + c2["retried_items"] > 0) == keep
    assert torch.equal(rgb, ref)
    b.close()
