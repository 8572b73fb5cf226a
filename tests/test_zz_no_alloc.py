"""The allocation-free local render (splx_render_partial_noalloc) against the allocating
splx_render_partial, through the C ABI, on two calls in a row.

That entry point serves callers that cannot allocate device memory (their HBM is held by
another allocator, or cudaMalloc's implicit synchronisation is not allowed in their loop);
its scratch is a fixed array shared by every call.  This file is collected last so that a
failure here does not hide the other GPU tests of a run that stops at the first failure.
"""
import numpy as np
import pytest

from paper_2606_18588_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _render_both(ctx, sc, cam, o):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    dev = to_device(sc)
    sub = subset_struct(dev, 0, sc.n, sc.sh_degree)
    ref = S.new_partial(cam.height, cam.width)
    S.render_partial(ctx, sub, cam, o, ref, keep_state=False)
    got = S.new_partial(cam.height, cam.width)
    for k in got:
        got[k].fill_(7)  # stale values must be overwritten
    S.render_partial_noalloc(sub, cam, o, got)
    torch.cuda.synchronize()
    return ref, got


def test_noalloc_matches_render_partial_twice_in_a_row():
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import PIXEL_TOL
    ctx = S.Context()
    cases = [
        (I.uniform_scene(20_000, 31, 3, log_scale_mu=-3.0),
         I.pinhole(300, 200, 60.0, (0.3, -0.2, -3.0), (0, 0, 0)), S.opts()),
        (I.cluster_scene(30_000, 32, 1),
         I.orbit_cameras(1, 33, [(211, 173)])[0], S.opts(tile=8)),
    ]
    for sc, cam, o in cases:  # two calls in a row, different scenes, cameras and tiles
        ref, got = _render_both(ctx, sc, cam, o)
        for k in ("rgb", "T", "depth"):
            err = float((ref[k] - got[k]).abs().max())
            assert err <= PIXEL_TOL, (k, err)
        assert torch.equal(ref["last"], got["last"])
    ctx.close()


def test_noalloc_rejects_oversize_requests():
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    sc = I.uniform_scene(65_537, 5, 0)
    cam = I.pinhole(64, 64, 60.0, (0, 0, -3), (0, 0, 0))
    dev = to_device(sc)
    out = S.new_partial(64, 64)
    with pytest.raises(S.SplxError) as e:
        S.render_partial_noalloc(subset_struct(dev, 0, sc.n, 0), cam, S.opts(), out)
    assert e.value.code == S.ERR_INVALID
    big = I.pinhole(8192, 8192, 60.0, (0, 0, -3), (0, 0, 0))  # 262144 tiles > 65536
    with pytest.raises(S.SplxError) as e:
        S.render_partial_noalloc(subset_struct(dev, 0, 100, 0), big, S.opts(), out)
    assert e.value.code == S.ERR_INVALID
