"""GPU parity of the forward path (through the C ABI) against the FP64 oracle.

Binning (cull, rectangle, depth key, per-tile sorted lists) must match bit for bit;
pixels within 1e-4 max-abs, and pixels in the oracle's ambiguity band within 1e-4 plus their
flip bound."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_18588_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2606_18588_gb300 import splx as S
    c = S.Context()
    yield c
    c.close()


def _cases():
    sc1, cam1 = I.plain_forward_case(0)
    sc2 = I.cluster_scene(20_000, 2, 3)
    cam2 = I.orbit_cameras(1, 3, [(333, 197)])[0]
    sc3 = I.uniform_scene(3000, 4, 1, log_scale_mu=-2.5)
    cam3 = I.pinhole(97, 61, 75.0, (0.4, -0.3, -2.2), (0, 0, 0))
    return {"plain_10k_sh0_256": (sc1, cam1), "cluster_20k_sh3_ragged": (sc2, cam2),
            "uniform_3k_sh1_large": (sc3, cam3)}


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tile", [16, 8, 32])
def test_binning_bit_exact(ctx, name, tile):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import decode_records, subset_struct, to_device
    sc, cam = CASES[name]
    dev = to_device(sc)
    p = S.new_partial(cam.height, cam.width)
    st = S.render_partial(ctx, subset_struct(dev, 0, sc.n, sc.sh_degree), cam, S.opts(tile=tile), p)
    ranges, keys, rec = st.export()
    vals = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    vis_g, rect_g, db_g = decode_records(rec)
    vis_o, rect_o, db_o = O.bin(sc, cam)
    assert np.array_equal(vis_g, vis_o)
    m = vis_o.astype(bool)
    assert np.array_equal(rect_g[m], rect_o[m])
    assert np.array_equal(db_g[m], db_o[m])
    start, lst = O.tile_lists(sc, cam, tile)
    assert vals.size == lst.size
    # every key carries its Gaussian's exact FP32 depth bits
    assert np.array_equal((keys >> np.uint64(32)).astype(np.uint32), db_o[vals])
    nt = start.size - 1
    assert ranges.shape[0] == nt
    for t in range(nt):
        a, b = int(start[t]), int(start[t + 1])
        ga, gb = int(ranges[t, 0]), int(ranges[t, 1])
        if b == a:
            assert gb <= ga
            continue
        assert np.array_equal(vals[ga:gb], lst[a:b].astype(np.uint32)), t
    st.close()


def test_binning_bit_exact_on_long_segments(ctx):
    """Tile lists of 5k and 40k entries (the two large-segment sorts), with many exactly
    equal depths so the index tie-break decides the order."""
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    rng = np.random.default_rng(17)
    n1, n2 = 40_000, 5_000
    m = np.zeros((n1 + n2, 3), np.float32)
    m[:n1, :2] = -0.433 + rng.uniform(-0.004, 0.004, (n1, 2))  # inside tile (1, 1)
    m[n1:, 0] = 0.433 + rng.uniform(-0.004, 0.004, n2)          # tile (2, 1)
    m[n1:, 1] = -0.433 + rng.uniform(-0.004, 0.004, n2)
    m[:, 2] = rng.choice(np.float32([-0.5, 0.0, 0.25]), n1 + n2)  # three depths only
    sc = I.Scene(m, np.full((n1 + n2, 3), -7.0, np.float32),
                 np.tile(np.float32([1, 0, 0, 0]), (n1 + n2, 1)),
                 np.zeros(n1 + n2, np.float32), np.zeros((n1 + n2, 1, 3), np.float32), 0)
    cam = I.pinhole(64, 64, 60.0, (0.0, 0.0, -3.0), (0.0, 0.0, 0.0))
    dev = to_device(sc)
    p = S.new_partial(64, 64)
    st = S.render_partial(ctx, subset_struct(dev, 0, sc.n, 0), cam, S.opts(tile=16), p)
    ranges, keys, _ = st.export()
    vals = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    start, lst = O.tile_lists(sc, cam, 16)
    seg = np.diff(start)
    assert seg.max() > 16384 and ((seg > 2048) & (seg <= 16384)).any()
    for t in range(start.size - 1):
        a, b = int(start[t]), int(start[t + 1])
        ga, gb = int(ranges[t, 0]), int(ranges[t, 1])
        assert gb - ga == b - a
        assert np.array_equal(vals[ga:gb], lst[a:b].astype(np.uint32)), t
    st.close()


@pytest.mark.parametrize("n", [2049, 3000, 4096, 4097, 8192, 8193, 12289])
def test_segment_sort_at_chunk_boundaries(ctx, n):
    """One tile's list of n keys around the lengths where the sort switches from one CTA
    to chunks (2048), fills a chunk (4096) and needs one more merge round (8192, 12288),
    with many equal depths so the index tie-break decides the order."""
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import to_device, subset_struct
    rng = np.random.default_rng(n)
    m = np.zeros((n, 3), np.float32)
    m[:, :2] = -0.433 + rng.uniform(-0.004, 0.004, (n, 2))  # inside tile (1, 1)
    m[:, 2] = rng.choice(np.float32([-0.5, -0.25, 0.0, 0.25]), n)
    sc = I.Scene(m, np.full((n, 3), -7.0, np.float32), np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
                 np.zeros(n, np.float32), np.zeros((n, 1, 3), np.float32), 0)
    cam = I.pinhole(64, 64, 60.0, (0.0, 0.0, -3.0), (0.0, 0.0, 0.0))
    p = S.new_partial(64, 64)
    st = S.render_partial(ctx, subset_struct(to_device(sc), 0, n, 0), cam, S.opts(tile=16), p)
    ranges, keys, _ = st.export()
    vals = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    start, lst = O.tile_lists(sc, cam, 16)
    assert np.diff(start).max() == n
    for t in range(start.size - 1):
        a, b = int(start[t]), int(start[t + 1])
        ga, gb = int(ranges[t, 0]), int(ranges[t, 1])
        assert gb - ga == b - a
        assert np.array_equal(vals[ga:gb], lst[a:b].astype(np.uint32)), t
    st.close()


@pytest.mark.parametrize("name", list(CASES))
def test_partial_render_matches_oracle(ctx, name):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import PIXEL_TOL, check_band, subset_struct, to_device
    sc, cam = CASES[name]
    dev = to_device(sc)
    o = S.opts()
    p = S.new_partial(cam.height, cam.width)
    st = S.render_partial(ctx, subset_struct(dev, 0, sc.n, sc.sh_degree), cam, o, p)
    ranges, keys, _ = st.export()
    vals = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    torch.cuda.synchronize()
    ref = O.render(sc, cam, O.opts(), bounds=True)
    amb, fb = ref["amb"], ref["flip"]
    check_band(p["rgb"].cpu().numpy(), ref["C"], amb, fb["C"], label=f"{name} C")
    check_band(p["T"].cpu().numpy(), ref["T"], amb, fb["T"], label=f"{name} T")
    check_band(p["depth"].cpu().numpy(), ref["D"], amb, fb["D"],
               tol=PIXEL_TOL * (1.0 + np.abs(ref["D"])), label=f"{name} D")
    ok = amb == 0
    # last blended Gaussian: GPU list position -> Gaussian index, exact off the guard band
    last = p["last"].cpu().numpy()
    H, W = cam.height, cam.width
    tw = (W + 15) // 16
    ty, tx = np.mgrid[0:H, 0:W]
    tiles = (ty // 16) * tw + (tx // 16)
    gid = np.where(last >= 0, vals[np.minimum(ranges[tiles, 0] + np.maximum(last, 0),
                                              max(vals.size - 1, 0))].astype(np.int64), -1)
    assert np.array_equal(gid[ok], ref["last"][ok])
    st.close()


def test_forward_bit_identical_across_tile_sizes(ctx):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    sc, cam = CASES["cluster_20k_sh3_ragged"]
    dev = to_device(sc)
    outs = []
    for tile in (8, 16, 32):
        p = S.new_partial(cam.height, cam.width)
        S.render_partial(ctx, subset_struct(dev, 0, sc.n, sc.sh_degree), cam, S.opts(tile=tile), p,
                         keep_state=False)
        torch.cuda.synchronize()
        outs.append({k: p[k].cpu().numpy() for k in ("rgb", "T", "depth")})
    for o in outs[1:]:
        for k in ("rgb", "T", "depth"):
            assert np.array_equal(o[k], outs[0][k]), k


def test_composite_matches_oracle_and_monolithic(ctx):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import PIXEL_TOL, check_band, render_view, to_device
    sc, off, _, cams = I.cluster_case(40_000, 5, 4, 1, [(320, 200)])
    cam = cams[0]
    dev = to_device(sc)
    o = S.opts()
    img, T, parts, states = render_view(ctx, dev, off, cam, o, sc.sh_degree)
    ref = O.render_view(sc, off, cam, O.opts(), separable=True, bounds=True)
    ok = ref["amb"] == 0
    fb = ref["flip"]
    check_band(img.cpu().numpy(), ref["image"], ref["amb"], fb["image"], label="composite image")
    check_band(T.cpu().numpy(), ref["T"], ref["amb"], fb["T"], label="composite T")
    for k, p in enumerate(parts):
        check_band(p["rgb"].cpu().numpy(), ref["Cp"][k], ref["amb"], fb["partC"][k],
                   label=f"partial {k} C")
        check_band(p["T"].cpu().numpy(), ref["Tp"][k], ref["amb"], fb["partT"][k],
                   label=f"partial {k} T")
    # composition alone: the oracle's Eq. 5 on the GPU's own partials (its band: near-tied
    # keys and the saturation cut, each with its exact effect as the bound)
    Cp = np.stack([p["rgb"].cpu().numpy() for p in parts]).astype(np.float64)
    Tp = np.stack([p["T"].cpu().numpy() for p in parts]).astype(np.float64)
    Dp = np.stack([p["depth"].cpu().numpy() for p in parts]).astype(np.float64)
    rc = O.composite(Cp, Tp, Dp, O.opts(), bounds=True)
    check_band(img.cpu().numpy(), rc["image"], rc["amb"], rc["flip"]["image"], tol=1e-5,
               label="Eq. 5 on the GPU partials")
    for s in states:
        s.close()
    # Eq. 5 == Eq. 2 on separable pixels: GPU composite vs GPU monolithic render, exact up
    # to FP32 rounding without termination ...
    from gpu_util import subset_struct
    o0 = S.opts(eps_T=0.0, eps_comp=0.0)
    img0, _, _, st0 = render_view(ctx, dev, off, cam, o0, sc.sh_degree, keep_state=False)
    mono0 = S.new_partial(cam.height, cam.width)
    S.render_partial(ctx, subset_struct(dev, 0, sc.n, sc.sh_degree), cam, o0, mono0,
                     keep_state=False)
    torch.cuda.synchronize()
    ref0 = O.render_view(sc, off, cam, O.opts(eps_T=0.0, eps_comp=0.0), separable=True)
    sep0 = (ref0["sep"] == 1) & (ref0["amb"] == 0)
    assert sep0.mean() > 0.5
    e0 = np.abs(img0.cpu().numpy() - mono0["rgb"].cpu().numpy()).max(axis=0)
    assert e0[sep0].max() <= 1e-5
    # ... and with termination within the bound of the stop rule: a render may stop with up
    # to eps/(1 - alpha_max) unabsorbed, at K+1 places (K local renders + the monolithic one)
    mono = S.new_partial(cam.height, cam.width)
    S.render_partial(ctx, subset_struct(dev, 0, sc.n, sc.sh_degree), cam, o, mono, keep_state=False)
    torch.cuda.synchronize()
    mono_ref = O.render(sc, cam, O.opts())
    sep = (ref["sep"] == 1) & ok & (mono_ref["amb"] == 0)
    K = len(off) - 1
    cmax = max(float(img0.max()), 1.0)
    bound = cmax * ((K + 1) * 1e-4 / (1.0 - 0.99) + 1e-4)
    e2 = np.abs(img.cpu().numpy() - mono["rgb"].cpu().numpy()).max(axis=0)
    assert e2[sep].max() <= bound


@pytest.mark.parametrize("W,H", [(1, 1), (17, 3), (5, 40)])
def test_tiny_and_ragged_images(ctx, W, H):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import check_band, subset_struct, to_device
    sc = I.uniform_scene(500, 9, 0, log_scale_mu=-2.0)
    cam = I.pinhole(W, H, 60.0, (0, 0, -3), (0, 0, 0))
    dev = to_device(sc)
    p = S.new_partial(H, W)
    S.render_partial(ctx, subset_struct(dev, 0, sc.n, 0), cam, S.opts(tile=8), p, keep_state=False)
    torch.cuda.synchronize()
    ref = O.render(sc, cam, O.opts(tile=8), bounds=True)
    # a handful of pixels: a single band pixel is allowed, checked against its bound
    check_band(p["rgb"].cpu().numpy(), ref["C"], ref["amb"], ref["flip"]["C"],
               budget=max(0.01, 1.0 / (W * H)), label=f"{W}x{H} C")


def test_empty_and_fully_culled_subsets(ctx):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    sc = I.uniform_scene(64, 1, 0)
    sc.means[:, 2] = -10.0  # all behind the camera at z = -3
    cam = I.pinhole(40, 30, 60.0, (0, 0, -3), (0, 0, 0))
    dev = to_device(sc)
    for lo, hi in ((0, 0), (0, 64)):
        p = S.new_partial(30, 40)
        S.render_partial(ctx, subset_struct(dev, lo, hi, 0), cam, S.opts(), p, keep_state=False)
        torch.cuda.synchronize()
        assert torch.all(p["T"] == 1.0) and torch.all(p["rgb"] == 0.0)
        assert torch.all(p["last"] == -1)


def test_invalid_arguments_are_rejected(ctx):
    from paper_2606_18588_gb300 import splx as S
    from gpu_util import subset_struct, to_device
    sc, cam = I.plain_forward_case(0, n=100)
    dev = to_device(sc)
    p = S.new_partial(cam.height, cam.width)
    with pytest.raises(S.SplxError) as e:
        S.render_partial(ctx, subset_struct(dev, 0, sc.n, 0), cam, S.opts(tile=12), p)
    assert e.value.code == S.ERR_INVALID
    bad = subset_struct(dev, 0, sc.n, 0)
    bad.quats = dev["quats"].data_ptr() + 4  # misaligned quaternion array
    with pytest.raises(S.SplxError):
        S.render_partial(ctx, bad, cam, S.opts(), p)
