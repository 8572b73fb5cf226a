"""Cross-boundary per-ray filtering (Sec. 8.1) on the GPU against the oracle: the batch
with the filter on renders the oracle's filtered images (pixels within 1e-4 outside the
ambiguity band) and their gradients (1e-3 relative L2), with and without saturation
skipping, and the filter does change the images of a k-d split cluster scene."""
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


@pytest.fixture(scope="module")
def case():
    return I.cluster_case(60_000, 13, 4, 3, [(160, 120), (200, 150), (96, 64)])


def _batch(ctx, dev, off, cams, deg, boxes, order=None):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct
    subs = [subset_struct(dev, int(off[k]), int(off[k + 1]), deg) for k in range(len(off) - 1)]
    b = S.Batch(ctx, subs, cams, S.opts())
    if boxes is not None:
        b.set_cross_filter(boxes)
    if order is not None:
        b.set_order(order)
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    torch.cuda.synchronize()
    assert b.status()[0] == S.OK
    return b, rgb


@pytest.mark.parametrize("skipping", [False, True])
def test_filtered_render_and_gradients_match_the_oracle(ctx, case, skipping):
    from gpu_util import GRAD_TOL, check_band, params_struct, rel_l2, to_device, zeros_like_params
    from paper_2606_18588_gb300.visibility import orders_for_views
    sc, off, boxes, cams = case
    K = len(off) - 1
    order = orders_for_views(boxes, cams) if skipping else None
    dev = to_device(sc)
    b, rgb = _batch(ctx, dev, off, cams, sc.sh_degree, boxes, order)
    dL = np.zeros(b.rgb_off[-1], np.float32)
    rng = np.random.default_rng(3)
    dls = []
    for v, c in enumerate(cams):
        ov = None if order is None else list(order[v])
        ref = O.render_view(sc, off, c, O.opts(), order=ov, cells=boxes, bounds=True)
        ok = ref["amb"] == 0
        got = b.views(rgb)[v].cpu().numpy()
        check_band(got, ref["image"], ref["amb"], ref["flip"]["image"],
                   label=f"filtered view {v} (skipping {skipping})")
        d = rng.standard_normal((3, c.height, c.width)) * ok[None]
        dL[b.rgb_off[v]:b.rgb_off[v + 1]] = d.reshape(-1)
        dls.append((d, ov))
    g = zeros_like_params(dev)
    b.backward(torch.from_numpy(dL).cuda(), None,
               [params_struct(g, int(off[k]), int(off[k + 1]), sc.sh_degree) for k in range(K)])
    torch.cuda.synchronize()
    b.close()
    g_ref = None
    for c, (d, ov) in zip(cams, dls):
        gv = O.backward_view(sc, off, c, d, None, O.opts(), order=ov, cells=boxes)
        g_ref = gv if g_ref is None else [x + y for x, y in zip(g_ref, gv)]
    errs = {k: rel_l2(g[k].cpu().numpy(), gr) for k, gr in zip(GROUPS, g_ref)}
    assert all(e <= GRAD_TOL for e in errs.values()), errs


def test_filter_changes_the_image_and_turns_off(ctx, case):
    from gpu_util import to_device
    sc, off, boxes, cams = case
    dev = to_device(sc)
    b1, rgb1 = _batch(ctx, dev, off, cams, sc.sh_degree, boxes)
    b0, rgb0 = _batch(ctx, dev, off, cams, sc.sh_degree, None)
    diff = (rgb1 - rgb0).abs()
    assert float(diff.max()) > 1e-2  # cross-boundary Gaussians were taken off some rays
    b1.set_cross_filter(None)
    b1.forward(rgb1)
    torch.cuda.synchronize()
    assert torch.equal(rgb1, rgb0)
    b1.close()
    b0.close()
