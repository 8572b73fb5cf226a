"""The 120M-Gaussian training-step workload (aerial city, K = 32 k-d subsets, a batch of 8
views at 1920x1080 sampled from 500 aerial cameras), generated cell by cell into device
memory and run in the launch configuration the benchmark times (tile 16, saturation
skipping and spatial visibility on).  Parity on seeded samples of tiles of two of the
views: the oracle sees the Gaussians that a conservative host bound lets reach a sampled
tile, in their global order (on the CPU the same oracle gives the same pixels for that
subset as for the whole scene), pixels within 1e-4 outside the ambiguity band and within
1e-4 plus the oracle's flip bound inside it, gradients
of a loss on the sampled tiles within 1e-3 relative L2, and exactly zero gradient for every
Gaussian the bound leaves out."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_18588_gb300 import inputs as I

from city_util import reach_tiles, tile_sample

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")
N, SEED, K = 120_000_000, 4, 32
SAMPLED = (0, 5)


def test_training_step_120m_k32_sampled_tiles():
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import _subset_structs, city_to_device
    from paper_2606_18588_gb300.visibility import orders_for_views
    from gpu_util import GRAD_TOL, check_band, params_struct, rel_l2

    lay = I.city_layout(N, SEED, K)
    pool = I.aerial_cameras(SEED)
    cams = [pool[i] for i in I.step_views(SEED, 0, len(pool))]
    order = orders_for_views(lay.boxes, cams)
    sample = {v: tile_sample(cams[v], 16, 31 + v) for v in SAMPLED}
    picked = []

    def keep_reaching(k, sc):
        keep = np.zeros(sc.n, bool)
        for v, (mask, _) in sample.items():
            keep |= reach_tiles(sc, cams[v], mask)
        idx = np.nonzero(keep)[0]
        picked.append((int(lay.offsets[k]) + idx, sc.take(idx)))

    dev = city_to_device(lay, on_cell=keep_reaching)
    gidx = np.concatenate([p[0] for p in picked])
    sub = I.Scene(*(np.concatenate([getattr(p[1], a) for p in picked]) for a in
                    ("means", "log_scales", "quats", "opacity_logits", "sh")), lay.sh_degree)
    sub_off = np.zeros(K + 1, np.int64)
    sub_off[1:] = np.cumsum([p[0].size for p in picked])
    assert 1000 < gidx.size < N // 100

    ctx = S.Context()
    b = S.Batch(ctx, _subset_structs(dev, lay.offsets, lay.sh_degree), cams, S.opts(tile=16))
    b.set_order(order)
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    torch.cuda.synchronize()
    code, pairs = b.status()
    assert code == S.OK and pairs > 0

    rng = np.random.default_rng(SEED)
    dL = np.zeros(b.rgb_off[-1], np.float32)
    dls = {}
    for v, (mask, pix) in sample.items():
        ov = list(order[v])
        ref = O.render_view(sub, sub_off, cams[v], O.opts(), tile_mask=mask, order=ov,
                            bounds=True)
        ok = pix & (ref["amb"] == 0)
        got = b.views(rgb)[v].cpu().numpy()
        check_band(got, ref["image"], ref["amb"], ref["flip"]["image"], where=pix, budget=0.02,
                   label=f"city view {v} image")
        assert ref["T"][pix].min() < 0.5  # the sampled tiles see geometry
        d = rng.standard_normal((3, cams[v].height, cams[v].width)) * ok[None]
        dL[b.rgb_off[v]:b.rgb_off[v + 1]] = d.reshape(-1)
        dls[v] = (d, mask, ov)

    g = {k: torch.zeros_like(t) for k, t in dev.items()}
    b.backward(torch.from_numpy(dL).cuda(), None,
               [params_struct(g, int(lay.offsets[k]), int(lay.offsets[k + 1]), lay.sh_degree)
                for k in range(K)])
    torch.cuda.synchronize()
    b.close()
    g_ref = None
    for v, (d, mask, ov) in dls.items():
        gv = O.backward_view(sub, sub_off, cams[v], d, None, O.opts(), tile_mask=mask, order=ov)
        g_ref = gv if g_ref is None else [a + c for a, c in zip(g_ref, gv)]
    gi = torch.from_numpy(gidx).cuda()
    errs = {}
    for name, gr in zip(GROUPS, g_ref):
        sel = g[name][gi]
        errs[name] = rel_l2(sel.cpu().numpy(), gr)
        assert int(torch.count_nonzero(g[name])) == int(torch.count_nonzero(sel)), name
    assert all(e <= GRAD_TOL for e in errs.values()), errs
