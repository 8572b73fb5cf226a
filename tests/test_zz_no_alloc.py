"""The allocation-free local render (splx_render_partial_noalloc) against the allocating
splx_render_partial, through the C ABI, on two calls in a row (bit for bit), its rejection of
oversize requests, and its pair-overflow status.

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


def _cases(S):
    return [
        (I.uniform_scene(20_000, 31, 3, log_scale_mu=-3.0),
         I.pinhole(300, 200, 60.0, (0.3, -0.2, -3.0), (0, 0, 0)), S.opts()),
        (I.cluster_scene(30_000, 32, 1),
         I.orbit_cameras(1, 33, [(211, 173)])[0], S.opts(tile=8)),
    ]


def test_noalloc_matches_render_partial_twice_in_a_row():
    """Both entry points run the same kernels on the same inputs, so the outputs agree bit
    for bit (the tolerance of the other GPU tests, 1e-4, is not needed here)."""
    from paper_2606_18588_gb300 import splx as S
    ctx = S.Context()
    for sc, cam, o in _cases(S):  # two calls in a row, different scenes, cameras and tiles
        ref, got = _render_both(ctx, sc, cam, o)
        for k in ("rgb", "T", "depth", "last"):
            assert torch.equal(ref[k], got[k]), k
    ctx.close()


def test_noalloc_reports_pair_overflow_then_renders_again():
    """60,000 large Gaussians on a 2048 x 2048 image at tile 8 stay within the Gaussian and
    tile limits but list more than 2^20 (Gaussian, tile) pairs: the call returns
    SPLX_ERR_CAPACITY, and the next call, within the limits, is again bit-identical to
    splx_render_partial."""
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    ctx = S.Context()
    sc = I.uniform_scene(60_000, 41, 0, log_scale_mu=-4.0)
    cam = I.pinhole(2048, 2048, 60.0, (0.0, 0.0, -3.0), (0, 0, 0))
    o = S.opts(tile=8)
    dev = to_device(sc)
    sub = subset_struct(dev, 0, sc.n, 0)
    ref = S.new_partial(cam.height, cam.width)
    st = S.render_partial(ctx, sub, cam, o, ref)
    _, keys, _ = st.export()
    st.close()
    assert keys.size > (1 << 20)  # the allocating path lists them all
    out = S.new_partial(cam.height, cam.width)
    with pytest.raises(S.SplxError) as e:
        S.render_partial_noalloc(sub, cam, o, out)
    assert e.value.code == S.ERR_CAPACITY
    sc2, cam2, o2 = _cases(S)[1]
    ref2, got2 = _render_both(ctx, sc2, cam2, o2)
    for k in ("rgb", "T", "depth", "last"):
        assert torch.equal(ref2[k], got2[k]), k
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
