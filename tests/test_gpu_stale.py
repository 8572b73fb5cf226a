"""Stale saturation state (splx_batch_set_stale): the pixels that one visit's composition
finds saturated leave the subsets behind at the view's next visit, rendered with one launch
per stage.  Parity with the oracle's render and backward under a given state and with its
re-evaluated state; a visit after an identical one equals the exact waves bit for bit;
a captured training step keeps it on the device."""
import numpy as np
import pytest

from oracle import oracle as O
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


def _batch(ctx, dev, sc, off, cams, order=None, planes=None, visibility=True):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct
    subs = [subset_struct(dev, int(off[k]), int(off[k + 1]), sc.sh_degree)
            for k in range(len(off) - 1)]
    b = S.Batch(ctx, subs, cams, S.opts())
    b.set_visibility(visibility)
    if order is not None:
        b.set_order(order)
    if planes is not None:
        b.set_stale(planes)
    return b


def _forward(b):
    from paper_2606_18588_gb300 import splx as S
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    T = torch.empty(b.total_pixels, device="cuda")
    b.forward(rgb, T)
    torch.cuda.synchronize()
    assert b.status()[0] == S.OK
    return rgb, T


def _grads(b, dev, off, deg, dL):
    from gpu_util import params_struct, zeros_like_params
    g = zeros_like_params(dev)
    b.backward(dL, None, [params_struct(g, int(off[k]), int(off[k + 1]), deg)
                          for k in range(len(off) - 1)])
    torch.cuda.synchronize()
    return g


def _planes(cams, fill=255):
    return [torch.full((c.height * c.width,), fill, dtype=torch.uint8, device="cuda") for c in cams]


@pytest.mark.parametrize("visibility", [True, False])
def test_a_visit_after_an_identical_one_renders_what_the_waves_render(ctx, visibility):
    # (with the visible regions on, partial planes outside them are never written and the
    # re-evaluation must skip them; off, every subset has a plane everywhere)
    from paper_2606_18588_gb300.visibility import orders_for_views
    from gpu_util import rel_l2, to_device
    sc, off, boxes, cams = I.cluster_case(120_000, 9, 8, 3, [(160, 120), (96, 64), (131, 77)])
    orders = orders_for_views(boxes, cams)
    dev = to_device(sc)
    full = _batch(ctx, dev, sc, off, cams, visibility=visibility)
    rgb_f, T_f = _forward(full)
    full.close()
    waves = _batch(ctx, dev, sc, off, cams, orders, visibility=visibility)
    rgb_w, T_w = _forward(waves)
    skipped_w = waves.counters()["skipped_items"]
    npx = int(rgb_w.numel())
    dL = torch.from_numpy(np.random.default_rng(3).standard_normal(npx).astype(np.float32)).cuda()
    g_w = _grads(waves, dev, off, sc.sh_degree, dL)
    waves.close()
    planes = _planes(cams)
    st = _batch(ctx, dev, sc, off, cams, orders, planes, visibility=visibility)
    # first visit: nothing pruned, so the render without skipping
    rgb_1, T_1 = _forward(st)
    assert torch.equal(rgb_1, rgb_f) and torch.equal(T_1, T_f)
    assert st.counters()["skipped_items"] == 0
    s1 = [p.clone() for p in planes]
    assert sum(int((p < 255).sum()) for p in s1) > 0
    # second visit: the first visit's state leaves out what the waves leave out
    rgb_2, T_2 = _forward(st)
    assert torch.equal(rgb_2, rgb_w) and torch.equal(T_2, T_w)
    assert st.counters()["skipped_items"] == skipped_w > 0
    for a, b in zip(s1, planes):  # and re-evaluates to the same state
        assert torch.equal(a, b)
    g_s = _grads(st, dev, off, sc.sh_degree, dL)
    for k in GROUPS:
        assert rel_l2(g_s[k].cpu().numpy(), g_w[k].cpu().numpy()) < 1e-5, k
    st.close()


def test_stale_render_and_state_match_the_oracle(ctx):
    from test_oracle_pins import _cam, _saturating_slabs
    from gpu_util import GRAD_TOL, band_share, check_band, rel_l2, to_device
    from paper_2606_18588_gb300.visibility import orders_for_views
    sc, off, boxes = _saturating_slabs(27, half_middle=True)
    cams = [_cam(64, 48), _cam(80, 56, eye=(0.3, -0.2, -3.2))]
    orders = orders_for_views(boxes, cams)
    rng = np.random.default_rng(8)
    states = []
    for c in cams:
        s = rng.choice(np.array([0, 1, 2, 3, 255], np.uint8), (c.height, c.width))
        s[:16, :16] = 1
        s[16:32, 16:32] = 0
        states.append(s)
    dev = to_device(sc)
    planes = [torch.from_numpy(s.reshape(-1).copy()).cuda() for s in states]
    b = _batch(ctx, dev, sc, off, cams, orders, planes)
    rgb, T = _forward(b)
    imgs = b.views(rgb)
    refs = [O.render_view(sc, off, c, O.opts(), order=list(orders[v]), sat=states[v], bounds=True)
            for v, c in enumerate(cams)]
    assert b.counters()["skipped_items"] == sum(int(r["skip"].sum()) for r in refs) > 0
    for v, (c, r) in enumerate(zip(cams, refs)):
        check_band(imgs[v].cpu().numpy(), r["image"], r["amb"], r["flip"]["image"],
                   label=f"view {v} image with a stale state")
        got = planes[v].cpu().numpy().reshape(c.height, c.width)
        amb = r["sat_amb"] != 0
        band_share(amb.astype(np.uint8), label=f"view {v} state re-evaluation")
        assert np.array_equal(got[~amb], r["sat"][~amb]), f"view {v} state"
        assert (r["sat"] < 255).sum() > 0
    # the backward of that render (the planes now hold the new states: the partials are
    # those of the render above, which the backward reads)
    c = cams[0]
    ok = (refs[0]["amb"] == 0).astype(np.float64)
    dLdC = rng.standard_normal((3, c.height, c.width)) * ok[None]
    dL = torch.zeros(b.rgb_off[-1], device="cuda")
    dL[: 3 * c.height * c.width] = torch.from_numpy(dLdC.reshape(-1).astype(np.float32)).cuda()
    g = _grads(b, dev, off, sc.sh_degree, dL)
    g_ref = O.backward_view(sc, off, c, dLdC, None, O.opts(), order=list(orders[0]), sat=states[0])
    errs = {k: rel_l2(g[k].cpu().numpy(), gr) for k, gr in zip(GROUPS, g_ref)}
    assert all(e <= GRAD_TOL for e in errs.values()), errs
    b.close()


def test_stale_state_in_a_captured_training_step(ctx):
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import BatchedStep
    from paper_2606_18588_gb300.visibility import orders_for_views
    from gpu_util import to_device
    sc, off, boxes, cams = I.cluster_case(60_000, 13, 4, 2, [(128, 96), (96, 80)])
    orders = orders_for_views(boxes, cams)
    tg = [torch.from_numpy(I.random_image(c.height, c.width, 30 + i)) for i, c in enumerate(cams)]
    dev = to_device(sc)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        st = BatchedStep(ctx, dev, off, sc.sh_degree, cams, tg, S.opts(), stream=s,
                         order=orders, stale=True)
        st.run()  # first visit: nothing pruned
        s.synchronize()
        first = [p.clone() for p in st.sat]
        assert sum(int((p < 255).sum()) for p in first) > 0
        st.capture()
        for _ in range(3):
            st.replay()
        s.synchronize()
        assert st.status()[0] == S.OK
        assert int(st.step_dev.item()) == 4
        assert all(torch.isfinite(t).all() for t in dev.values())
        assert sum(int((p < 255).sum()) for p in st.sat) > 0
        # new poses start the states over
        st.set_views(cams, orders)
        s.synchronize()
        assert all(bool((p == 255).all()) for p in st.sat)
    st.close()
