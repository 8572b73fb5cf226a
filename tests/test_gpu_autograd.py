"""Differentiation wrapper: train.Renderer as a torch.autograd.Function over the batch API.
Its forward is the oracle's image (pixels within 1e-4 outside the ambiguity band, within
1e-4 plus the oracle's flip bound inside it), the
.grad that loss.backward() leaves on the parameter tensors is the oracle's gradient of the
same loss (1e-3 relative L2 per group), a second backward accumulates as torch does, and
the total transmittance output carries no gradient."""
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


def test_renderer_forward_and_backward_match_the_oracle(ctx):
    from gpu_util import GRAD_TOL, check_band, rel_l2, to_device
    from paper_2606_18588_gb300.train import Renderer
    sc, off, _, cams = I.cluster_case(20_000, 31, 4, 2, [(120, 88), (72, 56)])
    params = {k: v.requires_grad_() for k, v in to_device(sc).items()}
    r = Renderer(ctx, params, off, sc.sh_degree, cams)
    rgb, T = r.render()
    assert rgb.requires_grad and not T.requires_grad
    # loss = sum(w * rgb), w seeded and zero on the oracle's ambiguity band
    rng = np.random.default_rng(5)
    w = torch.zeros_like(rgb)
    g_ref = None
    for v, (cam, img) in enumerate(zip(cams, r.views(rgb.detach()))):
        ref = O.render_view(sc, off, cam, O.opts(), bounds=True)
        ok = ref["amb"] == 0
        check_band(img.cpu().numpy(), ref["image"], ref["amb"], ref["flip"]["image"],
                   label=f"Renderer view {v}")
        wv = (rng.standard_normal((3, cam.height, cam.width)) * ok[None]).astype(np.float32)
        r.views(w)[v].copy_(torch.from_numpy(wv))
        gv = O.backward_view(sc, off, cam, wv.astype(np.float64), None, O.opts())
        g_ref = gv if g_ref is None else [a + b for a, b in zip(g_ref, gv)]
    (rgb * w).sum().backward()
    torch.cuda.synchronize()
    errs = {k: rel_l2(params[k].grad.cpu().numpy(), gr) for k, gr in zip(GROUPS, g_ref)}
    assert all(e <= GRAD_TOL for e in errs.values()), errs
    # a second render and backward adds to .grad, as for any torch leaf
    first = {k: params[k].grad.clone() for k in GROUPS}
    rgb2, _ = r.render()
    (rgb2 * w).sum().backward()
    torch.cuda.synchronize()
    for k in GROUPS:  # the atomics add in another order: equal up to FP32 rounding
        assert rel_l2(params[k].grad.cpu().numpy(), 2 * first[k].cpu().numpy()) <= 1e-5, k
    r.close()
