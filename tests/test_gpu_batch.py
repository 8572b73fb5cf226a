"""Batched V x K path (one launch per stage for all views and subsets) against the plain
per-view path, CUDA-graph replay, capacity overflow detection and the L1 loss."""
import numpy as np
import pytest

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
def scene():
    sc, off, _, cams = I.cluster_case(30_000, 11, 4, 3, [(200, 120), (96, 64), (131, 77)])
    return sc, off, cams


def _subsets(dev, off, deg):
    from gpu_util import subset_struct
    return [subset_struct(dev, int(off[k]), int(off[k + 1]), deg) for k in range(len(off) - 1)]


def _grads(g, off, deg):
    from gpu_util import params_struct
    return [params_struct(g, int(off[k]), int(off[k + 1]), deg) for k in range(len(off) - 1)]


def test_batch_forward_equals_plain_and_backward_matches(ctx, scene):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import backward_view, render_view, rel_l2, to_device, zeros_like_params
    sc, off, cams = scene
    dev = to_device(sc)
    o = S.opts()
    b = S.Batch(ctx, _subsets(dev, off, sc.sh_degree), cams, o)
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    T = torch.empty(b.total_pixels, device="cuda")
    b.forward(rgb, T)
    code, pairs = b.status()
    assert code == S.OK and pairs > 0
    rng = np.random.default_rng(0)
    dL = torch.from_numpy(rng.standard_normal(b.rgb_off[-1]).astype(np.float32)).cuda()
    g = zeros_like_params(dev)
    b.backward(dL, None, _grads(g, off, sc.sh_degree))
    torch.cuda.synchronize()
    g_plain = zeros_like_params(dev)
    for v, cam in enumerate(cams):
        img, Tv, parts, states = render_view(ctx, dev, off, cam, o, sc.sh_degree)
        assert torch.equal(b.views(rgb)[v], img)
        assert torch.equal(T[b.pix_off[v]:b.pix_off[v + 1]].view(cam.height, cam.width), Tv)
        gv = backward_view(ctx, dev, off, cam, o, sc.sh_degree, parts, states,
                           b.views(dL)[v].contiguous(), None)
        for k in GROUPS:
            g_plain[k] += gv[k]
        for s in states:
            s.close()
    for k in GROUPS:
        assert rel_l2(g[k].cpu().numpy(), g_plain[k].cpu().numpy()) < 1e-5, k
    b.close()


def test_graph_replay_is_identical(ctx, scene):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import to_device, zeros_like_params
    sc, off, cams = scene
    dev = to_device(sc)
    o = S.opts()
    b = S.Batch(ctx, _subsets(dev, off, sc.sh_degree), cams, o)
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    torch.cuda.synchronize()
    ref = rgb.clone()
    rgb.zero_()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        S.graph_begin(ctx, s)
        b.forward(rgb, stream=s)
        gr = S.graph_end(ctx, s)
        gr.launch(s)
    s.synchronize()
    assert torch.equal(rgb, ref)
    gr.close()
    b.close()


def test_graph_timing_ring_reads_every_replay(ctx, scene):
    """The timing ring: each back-to-back replay of a captured training step records the
    batch's kernel events into its own slot, every slot reads back (no host wait between
    the replays), and once the ring is removed the graph replays and times as before (its
    event nodes point at the captured events again)."""
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import BatchedStep
    from gpu_util import to_device
    sc, off, cams = scene
    dev = to_device(sc)
    s = torch.cuda.Stream()
    tg = [torch.from_numpy(I.random_image(c.height, c.width, 5 + i)) for i, c in enumerate(cams)]
    with torch.cuda.stream(s):
        st = BatchedStep(ctx, dev, off, sc.sh_degree, cams, tg, S.opts(), stream=s)
        st.batch.set_timing(True)
        st.run()
        s.synchronize()
        st.capture()
        for ring in (4, 3):  # a second ring replaces the first
            st.graph.set_timing_ring(ring)
            for _ in range(ring):
                st.replay()
            s.synchronize()
            for i in range(ring):
                t = st.batch.kernel_times(st.graph, i)
                assert all(v >= 0 for v in t.values())
                assert t["project"] > 0 and t["raster_fwd"] > 0 and t["raster_bwd"] > 0
        with pytest.raises(S.SplxError):
            st.batch.kernel_times(st.graph, ring)  # outside the ring
        st.graph.set_timing_ring(0)
        st.replay()
        s.synchronize()
        assert st.status()[0] == S.OK
        assert st.batch.kernel_times()["raster_bwd"] > 0
    st.close()


def test_capacity_overflow_is_reported_not_faulted(ctx, scene):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import to_device
    sc, off, cams = scene
    dev = to_device(sc)
    b = S.Batch(ctx, _subsets(dev, off, sc.sh_degree), cams, S.opts(), pair_capacity=1000)
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    code, pairs = b.status()
    assert code == S.ERR_CAPACITY and pairs > 1000
    ctx.device_status()  # clears the status word
    b.close()


def test_loss_l1_value_and_gradient(ctx):
    from paper_2606_18588_gb300 import splx as S
    rng = np.random.default_rng(1)
    a = rng.uniform(0, 1, 10007).astype(np.float32)
    t = rng.uniform(0, 1, 10007).astype(np.float32)
    t[:7] = a[:7]  # exact ties: zero gradient
    ad, td = torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda()
    loss = torch.empty(1, device="cuda")
    dL = torch.empty_like(ad)
    S.loss_l1(ctx, ad, td, loss, dL)
    torch.cuda.synchronize()
    np.testing.assert_allclose(loss.item(), np.abs(a.astype(np.float64) - t).mean(), rtol=1e-5)
    np.testing.assert_array_equal(dL.cpu().numpy(), (np.sign(a - t) / a.size).astype(np.float32))


def test_hbm_budget_is_enforced(ctx):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    small = S.Context(hbm_budget_bytes=1 << 16)
    sc, cam = I.plain_forward_case(0, n=5000)
    dev = to_device(sc)
    p = S.new_partial(cam.height, cam.width)
    with pytest.raises(S.SplxError) as e:
        S.render_partial(small, subset_struct(dev, 0, sc.n, 0), cam, S.opts(), p)
    assert e.value.code == S.ERR_BUDGET
    assert small.scratch_bytes == 0
    small.close()


def test_persistent_launch_shapes_agree(ctx, scene):
    # every (tile side, CTAs per SM) launch shape renders the same image bit for bit and
    # the same gradients up to the summation order of the atomics
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import rel_l2, to_device, zeros_like_params
    sc, off, cams = scene
    dev = to_device(sc)
    rng = np.random.default_rng(1)
    ref_rgb = ref_g = None
    for tile in (8, 16, 32):
        b = S.Batch(ctx, _subsets(dev, off, sc.sh_degree), cams, S.opts(tile=tile))
        fmax, bmax = b.max_ctas_per_sm()
        assert fmax >= 1 and bmax >= 1
        if ref_rgb is None:
            dL = torch.from_numpy(rng.standard_normal(b.rgb_off[-1]).astype(np.float32)).cuda()
        for c in (0, 1, 3, min(fmax, bmax)):
            b.set_launch(c)
            rgb = torch.empty(b.rgb_off[-1], device="cuda")
            b.forward(rgb)
            g = zeros_like_params(dev)
            b.backward(dL, None, _grads(g, off, sc.sh_degree))
            torch.cuda.synchronize()
            code, _ = b.status()
            assert code == S.OK
            if ref_rgb is None:
                ref_rgb, ref_g = rgb, g
                continue
            assert torch.equal(rgb, ref_rgb), (tile, c)
            for k in GROUPS:
                assert rel_l2(g[k].cpu().numpy(), ref_g[k].cpu().numpy()) < 1e-5, (tile, c, k)
        with pytest.raises(S.SplxError):
            b.set_launch(-1)
        b.close()


def test_autotuner_picks_a_timed_candidate(ctx, scene):
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.autotune import autotune
    from gpu_util import to_device
    sc, off, cams = scene
    dev = to_device(sc)
    npx = sum(3 * c.width * c.height for c in cams)
    target = torch.rand(npx, device="cuda")
    before = {k: v.clone() for k, v in dev.items()}
    r = autotune(ctx, dev, off, sc.sh_degree, cams, target, tiles=(8, 16), ctas=(0, 2), reps=2)
    assert len(r.table) == 4
    assert (r.tile, r.ctas_per_sm, r.ms) in [tuple(t) for t in r.table]
    assert r.ms == min(t[2] for t in r.table)
    for k in dev:  # the tuner never updates the parameters
        assert torch.equal(dev[k], before[k])


def test_spatial_visibility_changes_nothing(ctx, scene):
    # work items outside a subset's visible region are skipped and their partial planes
    # neither written nor read; images are bit-identical with the regions off and
    # gradients agree up to the order of the atomics
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import rel_l2, to_device, zeros_like_params
    sc, off, cams = scene
    dev = to_device(sc)
    rng = np.random.default_rng(8)
    out = {}
    for vis in (True, False):
        b = S.Batch(ctx, _subsets(dev, off, sc.sh_degree), cams, S.opts())
        b.set_visibility(vis)
        rgb = torch.empty(b.rgb_off[-1], device="cuda")
        T = torch.empty(b.total_pixels, device="cuda")
        b.forward(rgb, T)
        if vis:
            dL = torch.from_numpy(rng.standard_normal(b.rgb_off[-1]).astype(np.float32)).cuda()
        g = zeros_like_params(dev)
        b.backward(dL, None, _grads(g, off, sc.sh_degree))
        torch.cuda.synchronize()
        code, _ = b.status()
        assert code == S.OK
        out[vis] = (rgb, T, g, b.counters())
        b.close()
    assert out[True][3]["outside_items"] > 0 and out[False][3]["outside_items"] == 0
    assert torch.equal(out[True][0], out[False][0])
    assert torch.equal(out[True][1], out[False][1])
    for k in GROUPS:
        assert rel_l2(out[True][2][k].cpu().numpy(), out[False][2][k].cpu().numpy()) < 1e-5, k


def test_visible_pairs_are_the_oracles_kept_gaussians(ctx, scene):
    # splx_batch_visible counts the (view, Gaussian) pairs the projection kept: the
    # oracle's binning specification keeps the same Gaussians, bit for bit
    from paper_2606_18588_gb300 import splx as S
    from oracle import oracle as O
    from gpu_util import to_device
    sc, off, cams = scene
    dev = to_device(sc)
    b = S.Batch(ctx, _subsets(dev, off, sc.sh_degree), cams, S.opts())
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    b.forward(rgb)
    expect = sum(int(O.bin(sc, c)[0].astype(bool).sum()) for c in cams)
    assert b.visible() == expect > 0
    b.close()
