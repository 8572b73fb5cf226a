"""L1 + D-SSIM loss (Sec. 2 step 4) through the C ABI against the FP64 oracle: loss value
and image gradient, one image and a batch of views of uneven sizes."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2606_18588_gb300 import splx as S
    c = S.Context()
    yield c
    c.close()


def _check(loss, g, ref_loss, ref_g):
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss) + 1e-7, (loss, ref_loss)
    scale = np.abs(ref_g).max()
    assert np.abs(g - ref_g).max() <= 1e-4 * scale, (np.abs(g - ref_g).max(), scale)


@pytest.mark.parametrize("W,H,lam", [(70, 45, 0.2), (300, 200, 0.2), (33, 1, 0.5), (64, 64, 1.0)])
def test_loss_l1_dssim_single_image(ctx, W, H, lam):
    from paper_2606_18588_gb300 import splx as S
    rng = np.random.default_rng(W * 1000 + H)
    x = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1).astype(np.float32)  # correlated target
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    loss = torch.zeros(1, device="cuda")
    dL = torch.empty_like(xd)
    S.loss_l1_dssim(ctx, xd, yd, loss, dL, lam)
    torch.cuda.synchronize()
    ref_loss, ref_g = O.loss_l1_dssim([x], [y], lam)
    _check(float(loss.item()), dL.cpu().numpy(), ref_loss, ref_g[0])


def test_loss_l1_dssim_zero_weight_is_l1(ctx):
    from paper_2606_18588_gb300 import splx as S
    rng = np.random.default_rng(9)
    x = torch.rand(3, 40, 50, device="cuda")
    y = torch.rand(3, 40, 50, device="cuda")
    l0, l1 = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    g0, g1 = torch.empty_like(x), torch.empty_like(x)
    S.loss_l1_dssim(ctx, x, y, l0, g0, 0.0)
    S.loss_l1(ctx, x, y, l1, g1)
    torch.cuda.synchronize()
    assert abs(l0.item() - l1.item()) <= 1e-6
    assert torch.allclose(g0, g1, rtol=0, atol=1e-9)


def test_batch_loss_l1_dssim_over_views(ctx):
    from paper_2606_18588_gb300 import inputs as I
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    sc, off, _, cams = I.cluster_case(20_000, 4, 2, 3, [(131, 77), (64, 96), (200, 120)])
    dev = to_device(sc)
    subs = [subset_struct(dev, int(off[k]), int(off[k + 1]), sc.sh_degree) for k in range(2)]
    b = S.Batch(ctx, subs, cams, S.opts())
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    tgt = torch.rand_like(rgb)
    loss = torch.zeros(1, device="cuda")
    dL = torch.empty_like(rgb)
    b.loss_l1_dssim(rgb, tgt, loss, dL, 0.2)
    torch.cuda.synchronize()
    xs = [v.cpu().numpy() for v in b.views(rgb)]
    ys = [v.cpu().numpy() for v in b.views(tgt)]
    ref_loss, ref_g = O.loss_l1_dssim(xs, ys, 0.2)
    _check(float(loss.item()), dL.cpu().numpy(), ref_loss,
           np.concatenate([g.reshape(-1) for g in ref_g]))
    b.close()
