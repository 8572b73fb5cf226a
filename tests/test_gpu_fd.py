"""GPU gradients of the batched path against FP64 central finite differences (not against
the oracle's own adjoint), on the sub-scene the benchmark's workload names for it: the 200
Gaussians of the 10M-Gaussian K = 8 scene nearest the centre ray of its view 0, rendered at
128 x 128 from that view's pose, each kept in its k-d subset.

The finite differences come from the FP64 oracle's forward (h = 1e-7 max(1, |p|)); a
parameter whose +-h changes a discrete decision (visibility, rectangle, contributors,
subset order, clamp branches) is left out, and the loss weights are zero on the oracle's
ambiguity band.  Per parameter group the GPU gradient must lie within 1e-3 relative L2 of
the differences over the checked parameters."""
import os
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_18588_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_oracle_pins as P  # noqa: E402

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _sub_scene():
    w = I.WORKLOADS["batched_10m_k8"]
    sc, off, _, cams = I.cluster_case(w["n"], 3, w["K"], w["views"], w["sizes"], w["sh_degree"])
    c0 = cams[0]
    eye = c0.eye
    fwd = c0.R.astype(np.float64)[2]  # camera z axis in world coordinates
    rel = sc.means.astype(np.float64) - eye
    along = rel @ fwd
    dist = np.linalg.norm(rel - along[:, None] * fwd[None], axis=1)
    dist[along <= c0.near] = np.inf
    idx = np.sort(np.argpartition(dist, 200)[:200])
    member = np.searchsorted(off, idx, side="right") - 1
    kept = [k for k in range(len(off) - 1) if (member == k).any()]
    sub_off = np.concatenate([[0], np.cumsum([(member == k).sum() for k in kept])])
    cam = I.pinhole(128, 128, 60.0, eye, eye + fwd, c0.near)
    return sc.take(idx), sub_off, cam


def test_batched_gradients_match_fp64_finite_differences_on_200_gaussians():
    from gpu_util import GRAD_TOL, band_share, params_struct, rel_l2, subset_struct, to_device
    from gpu_util import zeros_like_params
    from paper_2606_18588_gb300 import splx as S
    sc, off, cam = _sub_scene()
    K = len(off) - 1
    o = O.opts()
    ref = O.render_view(sc, off, cam, o)
    assert ref["T"].min() < 0.5  # the sub-scene is in view
    band_share(ref["amb"], label="finite-difference sub-scene")
    rng = np.random.default_rng(23)
    wC = rng.standard_normal((3, cam.height, cam.width)) * (ref["amb"] == 0)[None]

    ctx = S.Context()
    dev = to_device(sc)
    subs = [subset_struct(dev, int(off[k]), int(off[k + 1]), sc.sh_degree) for k in range(K)]
    b = S.Batch(ctx, subs, [cam], S.opts(tile=16))
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    g = zeros_like_params(dev)
    b.backward(torch.from_numpy(wC.reshape(-1).astype(np.float32)).cuda(), None,
               [params_struct(g, int(off[k]), int(off[k + 1]), sc.sh_degree) for k in range(K)])
    torch.cuda.synchronize()
    assert b.status()[0] == S.OK
    b.close()
    ctx.close()

    base_sig = P._signature(sc, off, cam, o)
    arrays = list(sc.arrays())
    errs = {}
    for ai, name in enumerate(GROUPS):
        flat = arrays[ai].reshape(-1)
        gg = g[name].cpu().numpy().astype(np.float64).reshape(-1)
        fd_vals, gpu_vals = [], []
        for j in rng.choice(flat.size, size=min(flat.size, 40), replace=False):
            x0 = float(flat[j])
            h = 1e-7 * max(1.0, abs(x0))
            vals = []
            for sgn in (1, -1):
                sc2 = I.Scene(*[a.astype(np.float64).copy() for a in arrays], sc.sh_degree)
                sc2.arrays()[ai].reshape(-1)[j] = x0 + sgn * h
                if P._signature(sc2, off, cam, o) != base_sig:
                    break
                vals.append(float(np.sum(wC * O.render_view(sc2, off, cam, o)["image"])))
            if len(vals) < 2:
                continue
            fd_vals.append((vals[0] - vals[1]) / (2 * h))
            gpu_vals.append(gg[j])
        assert len(fd_vals) >= 25, (name, len(fd_vals))
        errs[name] = rel_l2(gpu_vals, fd_vals)
    print(f"[fd] GPU batched gradient vs FP64 central differences, rel L2 per group: {errs}")
    assert all(e <= GRAD_TOL for e in errs.values()), errs
