"""Adam fused into the projection adjoint (splx_batch_backward_adam) against the backward
into gradient arrays followed by the separate Adam pass (splx_batch_backward +
splx_step_device): bit-identical parameters and moments where the backward itself is
deterministic, close agreement on a clustered scene through a captured graph, and the
argument checks."""
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


def _tile_bound_case(sizes=(333, 400, 267), deg=3, seed=7, hidden=0):
    """Gaussians whose footprints lie inside one 16-pixel tile in each of two 128x128 views
    (the second view's principal point shifted by exactly one tile), so each (view,
    Gaussian) 2-D gradient is a single atomic add onto zero and the whole backward is
    deterministic.  Centres sit within 2 px of a tile centre; projected standard deviations
    are below 0.7 px before the 0.3 px^2 dilation, so 3-sigma footprints stay within 5 px
    of it.  The three subsets are contiguous with sizes that put subset boundaries inside
    128-Gaussian blocks.  The last `hidden` Gaussians lie behind both cameras (no view keeps
    them, so they have no gradient)."""
    rng = np.random.default_rng(seed)
    n = sum(sizes)
    f, c0 = 100.0, 64.0
    u = 8.0 + 16.0 * rng.integers(0, 8, n) + rng.uniform(-2.0, 2.0, n)
    v = 8.0 + 16.0 * rng.integers(0, 8, n) + rng.uniform(-2.0, 2.0, n)
    z = rng.uniform(4.5, 5.5, n)
    means = np.stack([(u - c0) * z / f, (v - c0) * z / f, z], 1).astype(np.float32)
    if hidden:
        means[n - hidden:, 2] = -means[n - hidden:, 2]
    log_scales = np.log(rng.uniform(0.01, 0.03, (n, 3))).astype(np.float32)
    q = rng.standard_normal((n, 4)).astype(np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(0.5, 1.0, n).astype(np.float32)
    nc = I.n_sh_coeffs(deg)
    sh = rng.normal(0.0, 0.5, (n, nc, 3)).astype(np.float32)
    sc = I.Scene(means, log_scales, q, logits, sh, deg)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    eye3, t0 = np.eye(3, dtype=np.float32), np.zeros(3, np.float32)
    cams = [I.Camera(eye3, t0, f, f, c0, c0, 128, 128),
            I.Camera(eye3, t0, f, f, c0 + 16.0, c0, 128, 128)]
    return sc, off, cams


def _train(ctx, sc, off, cams, tg, fused, steps, graph=False):
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import BatchedStep
    dev = {k: torch.from_numpy(np.ascontiguousarray(a)).cuda() for k, a in zip(GROUPS, sc.arrays())}
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        st = BatchedStep(ctx, dev, off, sc.sh_degree, cams, tg, S.opts(), stream=s,
                         fused_adam=fused)
        st.run()
        if graph:
            s.synchronize()
            st.capture()
            for _ in range(steps - 1):
                st.replay()
        else:
            for _ in range(steps - 1):
                st.run()
        s.synchronize()
        assert st.status()[0] == S.OK
    out = {"p": {k: t.clone() for k, t in dev.items()}, "m": {k: t.clone() for k, t in st.m.items()},
           "v": {k: t.clone() for k, t in st.v.items()}, "step": int(st.step_dev.item())}
    st.close()
    return out


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_fused_adam_is_bit_identical_where_the_backward_is_deterministic(ctx, deg):
    sc, off, cams = _tile_bound_case(deg=deg)
    tg = [torch.from_numpy(I.random_image(c.height, c.width, 40 + i)) for i, c in enumerate(cams)]
    a = _train(ctx, sc, off, cams, tg, fused=False, steps=3)
    a2 = _train(ctx, sc, off, cams, tg, fused=False, steps=3)
    for part in ("p", "m", "v"):  # the premise: this case's backward is deterministic
        for k in GROUPS:
            assert torch.equal(a[part][k], a2[part][k]), (part, k)
    b = _train(ctx, sc, off, cams, tg, fused=True, steps=3)
    assert a["step"] == b["step"] == 3
    moved = 0
    for part in ("p", "m", "v"):
        for k in GROUPS:
            assert torch.equal(a[part][k], b[part][k]), (part, k)
    for k in GROUPS:  # the steps did update every group
        moved += int((a["p"][k].cpu() != torch.from_numpy(getattr(sc, k))).any())
    assert moved == len(GROUPS)


def test_fused_adam_defers_blocks_without_gradients(ctx):
    # the last 300 Gaussians (two subsets) lie behind the cameras: the 128-Gaussian blocks
    # without any gradient go to the zero-gradient pass (one of them across the boundary of
    # the two hidden subsets, one partial at the end), the block that mixes visible and
    # hidden Gaussians stays in the fused epilogue; parameters and moments bit for bit those
    # of the separate Adam pass
    sizes = (333, 400, 267, 150, 150)
    sc, off, cams = _tile_bound_case(sizes=sizes, deg=3, seed=13, hidden=300)
    tg = [torch.from_numpy(I.random_image(c.height, c.width, 70 + i)) for i, c in enumerate(cams)]
    a = _train(ctx, sc, off, cams, tg, fused=False, steps=3)
    b = _train(ctx, sc, off, cams, tg, fused=True, steps=3)
    for part in ("p", "m", "v"):
        for k in GROUPS:
            assert torch.equal(a[part][k], b[part][k]), (part, k)
    # hidden Gaussians: zero gradient every step, so their moments stay zero and they stay put
    for k in GROUPS:
        assert not b["m"][k][1000:].any() and not b["v"][k][1000:].any(), k
        assert torch.equal(b["p"][k][1000:].cpu(), torch.from_numpy(getattr(sc, k)[1000:])), k


def test_fused_adam_with_an_empty_subset(ctx):
    # an empty subset between two others: its Adam entries are never touched, and the
    # 128-Gaussian blocks across the boundary still find their own subsets
    sc, off, cams = _tile_bound_case(sizes=(300, 0, 200), deg=2, seed=11)
    tg = [torch.from_numpy(I.random_image(c.height, c.width, 50 + i)) for i, c in enumerate(cams)]
    a = _train(ctx, sc, off, cams, tg, fused=False, steps=2)
    b = _train(ctx, sc, off, cams, tg, fused=True, steps=2)
    for part in ("p", "m", "v"):
        for k in GROUPS:
            assert torch.equal(a[part][k], b[part][k]), (part, k)


def test_fused_adam_agrees_on_a_clustered_scene_through_a_graph(ctx):
    sc, off, _, cams = I.cluster_case(30_000, 11, 4, 3, [(200, 120), (96, 64), (131, 77)])
    tg = [torch.from_numpy(I.random_image(c.height, c.width, 5 + i)) for i, c in enumerate(cams)]
    a = _train(ctx, sc, off, cams, tg, fused=False, steps=1)
    b = _train(ctx, sc, off, cams, tg, fused=True, steps=1)
    for k in GROUPS:
        p0 = torch.from_numpy(getattr(sc, k)).cuda().double()
        # the first moment is (1 - beta1) g: gradients equal up to atomic summation order
        ma, mb = a["m"][k].double(), b["m"][k].double()
        assert (ma - mb).norm() <= 1e-4 * ma.norm() + 1e-30, k
        # the first step moves each element by lr * g / (|g| + eps'): compare the moves
        da, db = a["p"][k].double() - p0, b["p"][k].double() - p0
        assert (da - db).norm() <= 1e-2 * da.norm(), k
    # several steps through a captured graph against the same number of eager ones
    a3 = _train(ctx, sc, off, cams, tg, fused=False, steps=3)
    b3 = _train(ctx, sc, off, cams, tg, fused=True, steps=3, graph=True)
    assert b3["step"] == 3
    for k in GROUPS:
        p0 = torch.from_numpy(getattr(sc, k)).cuda().double()
        da, db = a3["p"][k].double() - p0, b3["p"][k].double() - p0
        assert (da - db).norm() <= 2e-2 * da.norm(), k


def test_fused_adam_checks_its_arguments(ctx):
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import _subset_structs
    sc, off, cams = _tile_bound_case(sizes=(300, 200))
    dev = {k: torch.from_numpy(np.ascontiguousarray(a)).cuda() for k, a in zip(GROUPS, sc.arrays())}
    m = {k: torch.zeros_like(t) for k, t in dev.items()}
    v = {k: torch.zeros_like(t) for k, t in dev.items()}
    b = S.Batch(ctx, _subset_structs(dev, off, sc.sh_degree), cams, S.opts())
    rgb = torch.empty(b.rgb_off[-1], device="cuda")
    dL = torch.zeros_like(rgb)
    hp = S.adam_hp((1e-3,) * 6)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    ps = _subset_structs(dev, off, sc.sh_degree, mutable=True)
    ms = _subset_structs(m, off, sc.sh_degree, mutable=True)
    vs = _subset_structs(v, off, sc.sh_degree, mutable=True)
    with pytest.raises(S.SplxError) as e:  # before any forward
        b.backward_adam(dL, None, ps, ms, vs, hp, step)
    assert e.value.code == S.ERR_STATE
    b.forward(rgb)
    with pytest.raises(S.SplxError) as e:  # parameters that are not the batch's own
        b.backward_adam(dL, None, ms, ms, vs, hp, step)
    assert e.value.code == S.ERR_INVALID
    with pytest.raises(S.SplxError) as e:  # moments of the wrong size
        b.backward_adam(dL, None, ps, list(reversed(ms)), vs, hp, step)
    assert e.value.code == S.ERR_INVALID
    b.backward_adam(dL, None, ps, ms, vs, hp, step)
    torch.cuda.synchronize()
    assert int(step.item()) == 1
    # a zero loss gradient: every moment stays zero and no parameter moves
    for k in GROUPS:
        assert not m[k].any() and not v[k].any()
        assert torch.equal(dev[k].cpu(), torch.from_numpy(getattr(sc, k)))
    b.close()


def test_step_from_host_equals_the_captured_step(ctx):
    # the public step with host targets (forward graph, target upload on a copy stream,
    # then the update graph) trains exactly as the one-graph replay with device targets
    from paper_2606_18588_gb300 import splx as S
    from paper_2606_18588_gb300.train import BatchedStep
    sc, off, cams = _tile_bound_case()
    tg = [torch.from_numpy(I.random_image(c.height, c.width, 60 + i)) for i, c in enumerate(cams)]
    a = _train(ctx, sc, off, cams, tg, fused=True, steps=4, graph=True)
    dev = {k: torch.from_numpy(np.ascontiguousarray(x)).cuda() for k, x in zip(GROUPS, sc.arrays())}
    s = torch.cuda.Stream()
    host_t = torch.cat([t.reshape(-1) for t in tg]).pin_memory()
    host_loss = torch.empty(1).pin_memory()
    with torch.cuda.stream(s):
        st = BatchedStep(ctx, dev, off, sc.sh_degree, cams, None, S.opts(), stream=s)
        st.target.copy_(host_t.cuda())  # the first (eager) step's targets
        st.run()
        s.synchronize()
        st.capture_split()
        for _ in range(3):
            st.step_from_host(host_t, host_loss)
        s.synchronize()
        assert st.status()[0] == S.OK
    assert int(st.step_dev.item()) == 4
    for k in GROUPS:
        assert torch.equal(dev[k], a["p"][k]), k
        assert torch.equal(st.m[k], a["m"][k]) and torch.equal(st.v[k], a["v"][k]), k
    assert np.isfinite(host_loss.item()) and host_loss.item() > 0
    st.close()


def test_update_step_on_separately_allocated_subsets(ctx):
    # subsets in arrays of their own (not slices of one allocation): the update step takes
    # its block-by-block route, deferred blocks included; one step equals the backward into
    # gradient arrays followed by splx_step on each subset, bit for bit
    from paper_2606_18588_gb300 import splx as S
    sizes = (333, 400, 267, 150, 150)
    sc, off, cams = _tile_bound_case(sizes=sizes, deg=3, seed=17, hidden=300)
    K = len(sizes)
    lr = (1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3)

    def split():
        return [{k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k)[off[j]:off[j + 1]])).cuda()
                 for k in GROUPS} for j in range(K)]

    def run(fused):
        par = split()
        mom = [{k: torch.zeros_like(t) for k, t in d.items()} for d in par]
        vel = [{k: torch.zeros_like(t) for k, t in d.items()} for d in par]
        subs = [S.gaussians(*(d[k] for k in GROUPS), sc.sh_degree) for d in par]
        b = S.Batch(ctx, subs, cams, S.opts())
        rgb = torch.empty(b.rgb_off[-1], device="cuda")
        b.forward(rgb)
        tgt = torch.from_numpy(np.concatenate([I.random_image(c.height, c.width, 80 + i).reshape(-1)
                                               for i, c in enumerate(cams)])).cuda()
        loss = torch.zeros(1, device="cuda")
        dL = torch.empty_like(rgb)
        S.loss_l1(ctx, rgb, tgt, loss, dL)
        ps = [S.params(*(d[k] for k in GROUPS), sc.sh_degree) for d in par]
        ms = [S.params(*(d[k] for k in GROUPS), sc.sh_degree) for d in mom]
        vs = [S.params(*(d[k] for k in GROUPS), sc.sh_degree) for d in vel]
        if fused:
            step = torch.zeros(1, dtype=torch.int64, device="cuda")
            b.backward_adam(dL, None, ps, ms, vs, S.adam_hp(lr), step)
        else:
            gr = [{k: torch.zeros_like(t) for k, t in d.items()} for d in par]
            gs = [S.params(*(d[k] for k in GROUPS), sc.sh_degree) for d in gr]
            b.backward(dL, None, gs)
            for j in range(K):
                S.step(ctx, ps[j], gs[j], ms[j], vs[j], lr, 1)
        torch.cuda.synchronize()
        assert b.status()[0] == S.OK
        b.close()
        return par, mom, vel

    a, b = run(False), run(True)
    for x, y in zip(a, b):
        for dx, dy in zip(x, y):
            for k in GROUPS:
                assert torch.equal(dx[k], dy[k]), k
