"""Parity at the full sizes of the workloads, on seeded samples of tiles the oracle renders
one by one: the 1M-Gaussian K = 4 1920x1080 forward + backward, and the batched
10M-Gaussian K = 8 16-view step in the launch configuration the benchmark times (tile 16,
saturation skipping on).  Pixels within 1e-4 outside the oracle's ambiguity band and within
1e-4 plus the oracle's flip bound inside it, and gradients of a loss restricted to the
sampled tiles (zero on the band) within 1e-3 relative L2 per group."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_18588_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")
# Denser scenes evaluate more alphas per pixel near the threshold (about 200 per pixel on the
# 10M-Gaussian views), so their ambiguity band is wider; every band pixel is still checked
# against its flip bound.
FULLSIZE_BAND_BUDGET = 0.02


@pytest.fixture(scope="module")
def ctx():
    from paper_2606_18588_gb300 import splx as S
    c = S.Context()
    yield c
    c.close()


def _tile_sample(cam, n, seed, B=16):
    tw, th = (cam.width + B - 1) // B, (cam.height + B - 1) // B
    rng = np.random.default_rng(seed)
    mask = np.zeros(tw * th, np.uint8)
    mask[rng.choice(tw * th, size=n, replace=False)] = 1
    pix = np.zeros((th * B, tw * B), bool)
    pix.reshape(th, B, tw, B)[:] = mask.reshape(th, 1, tw, 1).astype(bool)
    return mask, pix[:cam.height, :cam.width]


def _parity(ctx, sc, off, cams, sample_views, n_tiles, seed, order=None):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import GRAD_TOL, check_band, params_struct, rel_l2, subset_struct, to_device
    from gpu_util import zeros_like_params
    dev = to_device(sc)
    K = len(off) - 1
    subs = [subset_struct(dev, int(off[k]), int(off[k + 1]), sc.sh_degree) for k in range(K)]
    b = S.Batch(ctx, subs, cams, S.opts(tile=16))
    if order is not None:
        b.set_order(order)
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    torch.cuda.synchronize()
    code, _ = b.status()
    assert code == S.OK
    dL = np.zeros(b.rgb_off[-1], np.float32)
    refs, dls = {}, {}
    rng = np.random.default_rng(seed)
    for v in sample_views:
        c = cams[v]
        mask, pix = _tile_sample(c, n_tiles, seed + v)
        ov = None if order is None else list(order[v])
        ref = O.render_view(sc, off, c, O.opts(), tile_mask=mask, order=ov, bounds=True)
        ok = pix & (ref["amb"] == 0)
        got = b.views(rgb)[v].cpu().numpy()
        check_band(got, ref["image"], ref["amb"], ref["flip"]["image"], where=pix,
                   budget=FULLSIZE_BAND_BUDGET, label=f"view {v} image")
        d = rng.standard_normal((3, c.height, c.width)) * ok[None]
        dls[v] = (d, mask, ov)
        dL[b.rgb_off[v]:b.rgb_off[v + 1]] = d.reshape(-1)
    g = zeros_like_params(dev)
    b.backward(torch.from_numpy(dL).cuda(), None,
               [params_struct(g, int(off[k]), int(off[k + 1]), sc.sh_degree) for k in range(K)])
    torch.cuda.synchronize()
    b.close()
    g_ref = None
    for v, (d, mask, ov) in dls.items():
        gv = O.backward_view(sc, off, cams[v], d, None, O.opts(), tile_mask=mask, order=ov)
        g_ref = gv if g_ref is None else [a + bb for a, bb in zip(g_ref, gv)]
    errs = {k: rel_l2(g[k].cpu().numpy(), gr) for k, gr in zip(GROUPS, g_ref)}
    assert all(e <= GRAD_TOL for e in errs.values()), errs
    return errs


def test_fwdbwd_1m_k4_1080p_sampled_tiles(ctx):
    sc, off, _, cams = I.cluster_case(1_000_000, 2, 4, 1, [(1920, 1080)])
    _parity(ctx, sc, off, cams, [0], 48, 11)


def test_batched_10m_k8_16_views_sampled_tiles(ctx):
    from paper_2606_18588_gb300.visibility import orders_for_views
    sc, off, boxes, cams = I.cluster_case(10_000_000, 3, 8, 16, [(1600, 1064), (1280, 720)])
    order = orders_for_views(boxes, cams)
    _parity(ctx, sc, off, cams, [0, 9], 16, 21, order=order)
