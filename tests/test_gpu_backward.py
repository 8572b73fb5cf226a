"""GPU parity of the backward (Eq. 6-7 and the chain to the Gaussian parameters) and of
Adam, through the C ABI, against the FP64 oracle."""
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


def _check_grads(ctx, sc, off, cam, use_dT, seed, tol=None):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import GRAD_TOL, backward_view, band_share, rel_l2, render_view, to_device
    tol = tol or GRAD_TOL
    dev = to_device(sc)
    o = S.opts()
    img, T, parts, states = render_view(ctx, dev, off, cam, o, sc.sh_degree)
    ref = O.render_view(sc, off, cam, O.opts())
    rng = np.random.default_rng(seed)
    H, W = cam.height, cam.width
    band_share(ref["amb"], label="backward view")
    ok = (ref["amb"] == 0).astype(np.float64)
    dLdC = rng.standard_normal((3, H, W)) * ok[None]
    dLdT = rng.standard_normal((H, W)) * ok if use_dT else None
    g_gpu = backward_view(ctx, dev, off, cam, o, sc.sh_degree, parts, states,
                          torch.from_numpy(dLdC.astype(np.float32)).cuda(),
                          None if dLdT is None else torch.from_numpy(dLdT.astype(np.float32)).cuda())
    g_ref = O.backward_view(sc, off, cam, dLdC, dLdT, O.opts())
    errs = {}
    for name, gr in zip(GROUPS, g_ref):
        errs[name] = rel_l2(g_gpu[name].cpu().numpy(), gr)
    for s in states:
        s.close()
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, errs
    return errs


def test_backward_single_subset_sh0(ctx):
    sc, cam = I.plain_forward_case(1, n=4000)
    _check_grads(ctx, sc, np.array([0, sc.n]), cam, False, 0)


def test_backward_k4_sh3_with_dT(ctx):
    sc, off, _, cams = I.cluster_case(8000, 7, 4, 1, [(160, 96)])
    _check_grads(ctx, sc, off, cams[0], True, 1)


def test_backward_k2_sh3_many_layers(ctx):
    sc = I.uniform_scene(6000, 8, 3, log_scale_mu=-2.6)
    perm, off, _ = I.kd_partition(sc.means, 2)
    sc = sc.take(perm)
    cam = I.pinhole(120, 90, 60.0, (0.2, -0.1, -3.0), (0, 0, 0))
    _check_grads(ctx, sc, off, cam, True, 2)


def test_adam_matches_oracle(ctx):
    from paper_2606_18588_gb300 import splx as S
    rng = np.random.default_rng(4)
    n, deg = 1001, 3
    shapes = {"means": (n, 3), "log_scales": (n, 3), "quats": (n, 4), "opacity_logits": (n,),
              "sh": (n, 16, 3)}
    P = {k: rng.standard_normal(s).astype(np.float32) for k, s in shapes.items()}
    Mo = {k: np.zeros(s) for k, s in shapes.items()}
    Vo = {k: np.zeros(s) for k, s in shapes.items()}
    Po = {k: v.astype(np.float64) for k, v in P.items()}
    dev = {k: torch.from_numpy(v).cuda() for k, v in P.items()}
    gd = {k: torch.zeros_like(v) for k, v in dev.items()}
    md = {k: torch.zeros_like(v) for k, v in dev.items()}
    vd = {k: torch.zeros_like(v) for k, v in dev.items()}
    lr = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 2.5e-3 / 20]
    st = lambda d: S.params(d["means"], d["log_scales"], d["quats"], d["opacity_logits"], d["sh"], deg)
    for step in range(1, 4):
        G = {k: rng.standard_normal(s).astype(np.float32) for k, s in shapes.items()}
        for k in G:
            gd[k].copy_(torch.from_numpy(G[k]))
        S.step(ctx, st(dev), st(gd), st(md), st(vd), lr, step, eps=1e-15)
        for i, k in enumerate(("means", "log_scales", "quats", "opacity_logits")):
            O.adam(Po[k].reshape(-1), G[k].astype(np.float64).reshape(-1), Mo[k].reshape(-1),
                   Vo[k].reshape(-1), lr[i], 0.9, 0.999, 1e-15, step)
        # SH: degree-0 coefficients and the rest take different learning rates
        for sl, l in ((np.s_[:, :1, :], lr[4]), (np.s_[:, 1:, :], lr[5])):
            p = np.ascontiguousarray(Po["sh"][sl]); m = np.ascontiguousarray(Mo["sh"][sl])
            v = np.ascontiguousarray(Vo["sh"][sl])
            O.adam(p.reshape(-1), np.ascontiguousarray(G["sh"][sl]).astype(np.float64).reshape(-1),
                   m.reshape(-1), v.reshape(-1), l, 0.9, 0.999, 1e-15, step)
            Po["sh"][sl], Mo["sh"][sl], Vo["sh"][sl] = p, m, v
    torch.cuda.synchronize()
    for k in shapes:
        np.testing.assert_allclose(dev[k].cpu().numpy(), Po[k], rtol=1e-5, atol=1e-6)
