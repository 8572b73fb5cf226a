"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test fixes a part of the oracle against a closed form, a library routine, brute
force or finite differences, chosen so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_18588_gb300 import inputs as I

Y00 = 0.5 / math.sqrt(math.pi)


def _scene(means, log_scales, quats, logits, rgb=None, sh=None, deg=0):
    n = len(means)
    if sh is None:
        sh = np.zeros((n, I.n_sh_coeffs(deg), 3), np.float32)
        sh[:, 0, :] = (np.asarray(rgb, np.float64) - 0.5) / Y00
    return I.Scene(np.asarray(means, np.float32).reshape(n, 3),
                   np.asarray(log_scales, np.float32).reshape(n, 3),
                   np.asarray(quats, np.float32).reshape(n, 4),
                   np.asarray(logits, np.float32).reshape(n),
                   np.asarray(sh, np.float32), deg)


def _cam(W=64, H=48, fov=60.0, eye=(0.0, 0.0, -3.0)):
    return I.pinhole(W, H, fov, eye, (0.0, 0.0, 0.0), 0.01)


def _logit(o):
    return math.log(o / (1.0 - o))


# --------------------------------------------------------------------------- exp spec
def test_exp_spec_within_3_ulp_of_exp():
    x = np.linspace(-20.0, 12.0, 200001).astype(np.float32)
    y = O.exp_spec(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(y - ref) / ulp) <= 3.0
    assert O.exp_spec(np.array([0.0], np.float32))[0] == 1.0


def test_log_spec_within_3_ulp_of_log():
    # the tile test's threshold 2 ln(o / (0.999 alpha_min)) takes arguments in [1, 256)
    x = np.concatenate([np.linspace(1.0, 256.0, 200001), np.geomspace(1.0, 1e30, 20001)])
    x = x.astype(np.float32)
    y = O.log_spec(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    ulp = np.spacing(np.maximum(ref, 1e-30).astype(np.float32)).astype(np.float64)
    big = ref > 1e-3  # near x = 1 the result is tiny: compare absolutely there
    assert np.max(np.abs(y - ref)[big] / ulp[big]) <= 3.0
    assert np.max(np.abs(y - ref)[~big]) <= 1e-9
    assert O.log_spec(np.array([1.0], np.float32))[0] == 0.0


# --------------------------------------------------------------------------- SH basis
def test_sh_basis_matches_scipy_real_harmonics():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(3)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    ref = []
    for l in range(4):
        for m in range(-l, l + 1):
            Y = sp.sph_harm_y(l, abs(m), theta, phi)  # complex, Condon-Shortley phase
            if m > 0:
                ref.append(math.sqrt(2.0) * Y.real)
            elif m < 0:
                ref.append(math.sqrt(2.0) * Y.imag)
            else:
                ref.append(Y.real)
    ref = np.stack(ref, axis=1)
    got = O.sh_basis(d)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_sh_basis_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    d = rng.standard_normal((20, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    g = O.sh_basis(d, grad=True)
    h = 1e-6
    for e in range(3):
        dp = d.copy(); dp[:, e] += h
        dm = d.copy(); dm[:, e] -= h
        fd = (O.sh_basis(dp) - O.sh_basis(dm)) / (2 * h)
        np.testing.assert_allclose(g[:, :, e], fd, atol=1e-7)


# --------------------------------------------------------------------------- closed forms
def _closed_form_image(cam, u, v, Sig, o, c, depth, r):
    """alpha-blend of one Gaussian with 2-D covariance Sig: C = c*alpha, T = 1-alpha."""
    H, W = cam.height, cam.width
    Q = np.linalg.inv(Sig)
    py, px = np.mgrid[0:H, 0:W]
    dx = px + 0.5 - u
    dy = py + 0.5 - v
    power = -0.5 * (Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy)
    alpha = np.minimum(0.99, o * np.exp(power))
    inside = (np.abs(px + 0.5 - u) <= r) & (np.abs(py + 0.5 - v) <= r)
    alpha = np.where(inside & (alpha >= 1.0 / 255.0), alpha, 0.0)
    return c[:, None, None] * alpha, 1.0 - alpha, depth * alpha


@pytest.mark.parametrize("case", ["iso", "aniso_rot", "offaxis", "offaxis_xz"])
def test_single_gaussian_closed_form(case):
    cam = _cam(64, 48)
    f = cam.fx
    o = 0.8
    rgb = np.array([0.9, 0.4, 0.1])
    z = 3.0
    if case == "iso":
        s = np.array([0.05, 0.05, 0.05]); mean = [0.0, 0.0, 0.0]; th = 0.0
    elif case == "aniso_rot":
        s = np.array([0.08, 0.02, 0.05]); mean = [0.0, 0.0, 0.0]; th = 0.7
    elif case == "offaxis":
        s = np.array([0.04, 0.04, 0.04]); mean = [0.3, 0.0, 0.0]; th = 0.0
    else:
        s = np.array([0.15, 0.01, 0.01]); mean = [0.8, 0.0, 0.0]; th = 0.0
    q = [math.cos(th / 2), 0.0, 0.0, math.sin(th / 2)]  # rotation about the optical axis
    if case == "offaxis_xz":
        q = [math.cos(math.pi / 8), 0.0, math.sin(math.pi / 8), 0.0]  # 45 deg about y
    sc = _scene([mean], [np.log(s)], [q], [_logit(o)], rgb=[rgb])
    sf = np.exp(np.asarray(sc.log_scales[0], np.float64))  # the exact stored scale
    x = float(sc.means[0, 0])
    # Sigma2D = J R diag(s^2) R^T J^T + 0.3 I; the camera axes are the world axes here.
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    if case == "offaxis_xz":
        c4 = math.cos(math.pi / 4)
        Rz = np.array([[c4, 0, c4], [0, 1, 0], [-c4, 0, c4]])
    Sig3 = Rz @ np.diag(sf ** 2) @ Rz.T
    J = np.array([[f / z, 0.0, -f * x / z ** 2], [0.0, f / z, 0.0]])
    Sig = J @ Sig3 @ J.T + 0.3 * np.eye(2)
    u = f * x / z + cam.cx
    v = cam.cy
    lam = 0.5 * (Sig[0, 0] + Sig[1, 1]) + math.sqrt(max(0.1, (0.5 * (Sig[0, 0] - Sig[1, 1])) ** 2
                                                      + Sig[0, 1] ** 2))
    r = math.ceil(3.0 * math.sqrt(lam))
    C, T, D = _closed_form_image(cam, u, v, Sig, o, rgb, z, r)
    got = O.render(sc, cam, O.opts(tile=16, eps_T=0.0, eps_comp=0.0))
    np.testing.assert_allclose(got["C"], C, atol=1e-6)
    np.testing.assert_allclose(got["T"], T, atol=1e-6)
    np.testing.assert_allclose(got["D"], D, atol=1e-5)
    # the FP64 projection itself (conic = Sigma2D^{-1}, mean, depth)
    pr = O.project(sc, cam)[0]
    Q = np.linalg.inv(Sig)
    np.testing.assert_allclose(pr[[0, 1]], [u, v], rtol=1e-6)
    np.testing.assert_allclose(pr[[2, 3, 4]], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-5)
    np.testing.assert_allclose(pr[9], z, rtol=1e-6)


def test_colour_dc_only_is_y00_times_dc_plus_half():
    cam = _cam()
    rng = np.random.default_rng(0)
    rgb = rng.uniform(0, 1, (5, 3))
    sc = _scene(rng.uniform(-0.5, 0.5, (5, 3)), np.full((5, 3), -3.0), [[1, 0, 0, 0]] * 5,
                np.zeros(5), rgb=rgb)
    pr = O.project(sc, cam)
    np.testing.assert_allclose(pr[:, 6:9], rgb, atol=1e-6)


def test_colour_degree1_closed_form():
    # degree-1 colour = Y00*dc + 0.5 + k1*(-y*c1 + z*c2 - x*c3) at the unit viewing direction
    cam = _cam()
    sh = np.zeros((1, 4, 3), np.float32)
    sh[0, 1] = [0.3, 0.0, 0.0]; sh[0, 2] = [0.0, 0.2, 0.0]; sh[0, 3] = [0.0, 0.0, -0.25]
    sc = _scene([[0.4, -0.3, 0.5]], [[-3, -3, -3]], [[1, 0, 0, 0]], [0.0], sh=sh, deg=1)
    d = sc.means[0].astype(np.float64) - cam.eye
    d /= np.linalg.norm(d)
    k1 = math.sqrt(3.0 / (4.0 * math.pi))
    want = 0.5 + np.array([-k1 * d[1] * 0.3, k1 * d[2] * 0.2, -k1 * d[0] * -0.25])
    np.testing.assert_allclose(O.project(sc, cam)[0, 6:9], np.maximum(want, 0.0), atol=1e-7)


# --------------------------------------------------------------------------- brute force
def _brute_force(sc, cam, eps_T=1e-4, amin=1.0 / 255.0, amax=0.99):
    """Per pixel: gather every visible Gaussian whose rectangle holds it, order by
    (FP32 depth bits, index), blend literally.  No tiles, no per-tile lists."""
    vis, rect, db = O.bin(sc, cam)
    pr = O.project(sc, cam)
    H, W = cam.height, cam.width
    C = np.zeros((3, H, W)); T = np.ones((H, W)); D = np.zeros((H, W))
    order = sorted([i for i in range(sc.n) if vis[i]], key=lambda i: (int(db[i]), i))
    for py in range(H):
        for px in range(W):
            t = 1.0
            for i in order:
                x0, x1, y0, y1 = rect[i]
                if not (x0 <= px <= x1 and y0 <= py <= y1):
                    continue
                u, v, A, B, Cc, o = pr[i, :6]
                dx, dy = px + 0.5 - u, py + 0.5 - v
                power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy
                if power > 0:
                    continue
                a = min(amax, o * math.exp(power))
                if a < amin:
                    continue
                if t * (1 - a) < eps_T:
                    break
                C[:, py, px] += pr[i, 6:9] * a * t
                D[py, px] += pr[i, 9] * a * t
                t *= 1 - a
            T[py, px] = t
    return C, T, D


@pytest.mark.parametrize("n,seed,tile", [(1, 0, 8), (5, 1, 8), (20, 2, 16), (20, 3, 8)])
def test_render_matches_brute_force(n, seed, tile):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.4, 0.4, (n, 3))
    if n >= 5:
        means[1] = means[0]            # equal depth: exercises the index tie-break
    sc = _scene(means, rng.normal(-2.8, 0.4, (n, 3)), rng.standard_normal((n, 4)),
                rng.normal(1.0, 1.0, n), rgb=rng.uniform(0, 1, (n, 3)))
    cam = _cam(40, 32)
    Cb, Tb, Db = _brute_force(sc, cam)
    got = O.render(sc, cam, O.opts(tile=tile))
    np.testing.assert_allclose(got["C"], Cb, atol=1e-12)
    np.testing.assert_allclose(got["T"], Tb, atol=1e-12)
    np.testing.assert_allclose(got["D"], Db, atol=1e-12)


def test_tile_culling_drops_only_pairs_below_alpha_min():
    # every (Gaussian, tile) pair of the rectangle that the lists omit must have
    # alpha < alpha_min at every pixel centre it shares with the tile (FP64)
    sc, cam = I.plain_forward_case(6, n=1500)
    vis, rect, db = O.bin(sc, cam)
    pr = O.project(sc, cam)
    B = 16
    start, lst = O.tile_lists(sc, cam, B)
    tw = (cam.width + B - 1) // B
    listed = set()
    for t in range(start.size - 1):
        for g in lst[start[t]:start[t + 1]]:
            listed.add((int(g), t))
    culled = 0
    for g in np.nonzero(vis)[0]:
        x0, x1, y0, y1 = rect[g]
        u, v, A, Bc, Cc, o = pr[g, :6]
        for ty in range(y0 // B, y1 // B + 1):
            for tx in range(x0 // B, x1 // B + 1):
                if (int(g), ty * tw + tx) in listed:
                    continue
                culled += 1
                px = np.arange(max(tx * B, x0), min(tx * B + B - 1, x1) + 1) + 0.5 - u
                py = np.arange(max(ty * B, y0), min(ty * B + B - 1, y1) + 1) + 0.5 - v
                X, Y = np.meshgrid(px, py)
                alpha = o * np.exp(-0.5 * (A * X * X + Cc * Y * Y) - Bc * X * Y)
                assert alpha.max() < 1.0 / 255.0, (g, tx, ty, alpha.max())
    assert culled > 0.05 * len(listed)  # the culling does remove a real share of pairs


def test_tile_culling_is_the_box_maximum_of_alpha():
    # brute force: the largest alpha over the box of shared pixel centres (its boundary
    # sampled densely, its interior only through the mean) decides each pair; pairs
    # clearly above 0.999 alpha_min are listed, pairs clearly below are not
    sc, cam = I.plain_forward_case(7, n=800)
    vis, rect, db = O.bin(sc, cam)
    pr = O.project(sc, cam)
    B = 16
    start, lst = O.tile_lists(sc, cam, B)
    tw = (cam.width + B - 1) // B
    listed = {(int(g), t) for t in range(start.size - 1) for g in lst[start[t]:start[t + 1]]}
    s = np.linspace(0.0, 1.0, 4001)
    thr = 0.999 / 255.0
    checked = 0
    for g in np.nonzero(vis)[0]:
        x0, x1, y0, y1 = rect[g]
        u, v, A, Bc, Cc, o = pr[g, :6]
        for ty in range(y0 // B, y1 // B + 1):
            for tx in range(x0 // B, x1 // B + 1):
                xa, xb = max(tx * B, x0) + 0.5 - u, min(tx * B + B - 1, x1) + 0.5 - u
                ya, yb = max(ty * B, y0) + 0.5 - v, min(ty * B + B - 1, y1) + 0.5 - v
                if xa <= 0 <= xb and ya <= 0 <= yb:
                    qmin = 0.0
                else:
                    ex = np.concatenate([xa + (xb - xa) * s, xa + (xb - xa) * s,
                                         np.full_like(s, xa), np.full_like(s, xb)])
                    ey = np.concatenate([np.full_like(s, ya), np.full_like(s, yb),
                                         ya + (yb - ya) * s, ya + (yb - ya) * s])
                    qmin = np.min(A * ex * ex + 2.0 * Bc * ex * ey + Cc * ey * ey)
                amax = o * np.exp(-0.5 * qmin)
                key = (int(g), ty * tw + tx)
                if amax > thr * (1 + 1e-4):
                    assert key in listed, (g, tx, ty, amax)
                    checked += 1
                elif amax < thr * (1 - 1e-4):
                    assert key not in listed, (g, tx, ty, amax)
                    checked += 1
    assert checked > 500


def test_tile_lists_invariants_and_tile_size_independence():
    sc, cam = I.plain_forward_case(5, n=2000)
    vis, rect, db = O.bin(sc, cam)
    ref = None
    for B in (8, 16, 32):
        start, lst = O.tile_lists(sc, cam, B)
        tw = (cam.width + B - 1) // B
        expect = sum((r[1] // B - r[0] // B + 1) * (r[3] // B - r[2] // B + 1)
                     for r, v in zip(rect, vis) if v)
        assert 0 < lst.size <= expect
        for t in range(start.size - 1):
            seg = lst[start[t]:start[t + 1]]
            tx, ty = t % tw, t // tw
            for g in seg:
                x0, x1, y0, y1 = rect[g]
                assert x0 // B <= tx <= x1 // B and y0 // B <= ty <= y1 // B
            keys = [(int(db[g]), int(g)) for g in seg]
            assert keys == sorted(keys)
        out = O.render(sc, cam, O.opts(tile=B))
        if ref is None:
            ref = out
        else:
            for k in ("C", "T", "D", "last", "ncontrib"):
                assert np.array_equal(out[k], ref[k]), k


def test_blend_identity_sum_alpha_T_equals_one_minus_T():
    # with every colour equal to 1, C = sum_i alpha_i T_i = 1 - T exactly (Eq. 2-4)
    sc, cam = I.plain_forward_case(7, n=3000)
    sc.sh[:, 0, :] = np.float32(0.5 / Y00)
    out = O.render(sc, cam)
    for ch in range(3):
        np.testing.assert_allclose(out["C"][ch], 1.0 - out["T"], atol=1e-12)
    assert out["T"].min() >= 0.0 and out["T"].max() <= 1.0


def test_nearplane_and_degenerate_culls():
    cam = _cam()
    sc = _scene([[0, 0, -3.0 + 0.005], [0, 0, -3.0 + 0.02], [0, 0, 0.0], [5e3, 0, 0.0]],
                [[-3] * 3, [-3] * 3, [-3] * 3, [-3] * 3],
                [[1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 0], [1, 0, 0, 0]], [0, 0, 0, 0],
                rgb=[[1, 1, 1]] * 4)
    vis, rect, db = O.bin(sc, cam)
    assert list(vis) == [0, 1, 0, 0]  # behind near, kept, zero quaternion, off-image


# --------------------------------------------------------------------------- composite
def _slab_scene(seed, K=3, per=40):
    """K groups at disjoint depth slabs with a gap far above 3 sigma: separable pixels."""
    rng = np.random.default_rng(seed)
    means, ls = [], []
    for k in range(K):
        m = rng.uniform(-0.5, 0.5, (per, 3))
        m[:, 2] = -0.8 + 0.8 * k + rng.uniform(-0.15, 0.15, per)
        means.append(m)
        ls.append(rng.normal(-3.2, 0.2, (per, 3)))
    n = K * per
    sc = _scene(np.concatenate(means), np.concatenate(ls), rng.standard_normal((n, 4)),
                rng.normal(0.5, 1.0, n), rgb=rng.uniform(0, 1, (n, 3)))
    offsets = np.arange(K + 1) * per
    return sc, offsets


def test_composite_equals_monolithic_on_separable_scene():
    sc, off = _slab_scene(11)
    cam = _cam(48, 40)
    o = O.opts(eps_T=0.0, eps_comp=0.0)
    comp = O.render_view(sc, off, cam, o)
    mono = O.render_view(sc, np.array([0, sc.n]), cam, o)
    np.testing.assert_allclose(comp["image"], mono["image"], atol=1e-12)
    np.testing.assert_allclose(comp["T"], mono["T"], atol=1e-12)
    # a shuffled subset order must give the same image: order comes from the depth keys
    perm = [2, 0, 1]
    idx = np.concatenate([np.arange(off[k], off[k + 1]) for k in perm])
    sc2 = sc.take(idx)
    comp2 = O.render_view(sc2, off, cam, o)
    np.testing.assert_allclose(comp2["image"], mono["image"], atol=1e-12)


def test_composite_termination_bound():
    # A render stops before the Gaussian that would take T below eps, so it can stop with
    # T < eps / (1 - alpha_max) left; composite (K local cuts + the eps_comp cut) and the
    # exact render therefore differ by at most (K*eps/(1-alpha_max) + eps_comp) * max c.
    sc, off = _slab_scene(12)
    sc.opacity_logits[:] = 3.0
    cam = _cam(48, 40)
    exact = O.render_view(sc, np.array([0, sc.n]), cam, O.opts(eps_T=0.0, eps_comp=0.0))
    comp = O.render_view(sc, off, cam, O.opts(eps_T=1e-4, eps_comp=1e-4))
    K = len(off) - 1
    cmax = max(1.0, float(O.project(sc, cam)[:, 6:9].max()))
    err = np.abs(comp["image"] - exact["image"]).max()
    assert err <= cmax * (K * 1e-4 / (1 - 0.99) + 1e-4)
    # with the stop rule switched off the two agree to rounding
    comp0 = O.render_view(sc, off, cam, O.opts(eps_T=0.0, eps_comp=0.0))
    assert np.abs(comp0["image"] - exact["image"]).max() <= 1e-12


def test_composite_single_subset_is_identity_plus_background():
    rng = np.random.default_rng(2)
    Cp = rng.uniform(0, 0.5, (1, 3, 8, 8)); Tp = rng.uniform(0, 1, (1, 8, 8))
    Dp = rng.uniform(1, 2, (1, 8, 8))
    out = O.composite(Cp, Tp, Dp, O.opts(eps_comp=0.0, bg=(0.1, 0.2, 0.3)))
    np.testing.assert_allclose(out["image"], Cp[0] + np.array([0.1, 0.2, 0.3])[:, None, None] * Tp[0])
    np.testing.assert_allclose(out["T"], Tp[0])


def test_composite_is_the_over_operator_in_key_order():
    # (C,T) over (C',T') = (C + T C', T T'), applied in increasing D/(1-T); associative
    rng = np.random.default_rng(5)
    K, H, W = 4, 6, 7
    Tp = rng.uniform(0.05, 0.95, (K, H, W))
    Cp = rng.uniform(0, 1, (K, 3, H, W)) * (1 - Tp)[:, None]
    z = rng.uniform(1, 10, (K, H, W))
    Dp = z * (1 - Tp)
    out = O.composite(Cp, Tp, Dp, O.opts(eps_comp=0.0))
    order = np.argsort(z, axis=0, kind="stable")
    for py in range(H):
        for px in range(W):
            ms = order[:, py, px]
            # right fold
            c, t = np.zeros(3), 1.0
            for m in ms[::-1]:
                c = Cp[m, :, py, px] + Tp[m, py, px] * c
                t = Tp[m, py, px] * t
            np.testing.assert_allclose(out["image"][:, py, px], c, atol=1e-12)
            np.testing.assert_allclose(out["T"][py, px], t, atol=1e-12)


def test_kd_partition_convex_boxes_and_balance():
    sc = I.cluster_scene(4096, 3, 0)
    perm, off, boxes = I.kd_partition(sc.means, 8)
    assert sorted(perm.tolist()) == list(range(4096))
    assert np.all(np.diff(off) == 512)
    m = sc.means[perm].astype(np.float64)
    for k in range(8):
        seg = m[off[k]:off[k + 1]]
        lo, hi = boxes[k]
        assert np.all(seg >= lo - 1e-9) and np.all(seg <= hi + 1e-9)
        assert np.all(np.isinf(lo[1])) and np.all(np.isinf(hi[1]))  # y is never split


# --------------------------------------------------------------------------- finite differences
def _signature(sc, off, cam, o):
    vis, rect, db = O.bin(sc, cam)
    parts = []
    for k in range(len(off) - 1):
        r = O.render(sc.subset(off[k], off[k + 1]), cam, o)
        parts.append((r["last"].copy(), r["ncontrib"].copy()))
    v = O.render_view(sc, off, cam, o)
    key = np.where(v["Tp"] < 1, v["Dp"] / np.maximum(1 - v["Tp"], 1e-300), np.inf)
    order = np.argsort(key, axis=0, kind="stable")
    flags, ncl = O.branch_stats(sc, off, cam, o)
    return (vis.tobytes(), rect.tobytes(), b"".join(a.tobytes() + b.tobytes() for a, b in parts),
            order.tobytes(), flags.tobytes(), ncl.tobytes())


def _loss(sc, off, cam, o, wC, wT):
    v = O.render_view(sc, off, cam, o)
    return float(np.sum(wC * v["image"]) + np.sum(wT * v["T"]))


# The four Gaussians of the finite-difference scene that drive the adjoint's clamp branches
# (camera-space mean, log-scale, logit, colour; see _fd_scene).
FD_SIDE_X, FD_SIDE_Y, FD_OPAQUE, FD_DARK = range(4)


def _fd_scene(deg, seed):
    """24 random Gaussians around the origin, seen from 2.2 away by a 40 x 36 camera, plus
    four placed (in camera space) so that each clamp of the adjoint is active:
    - FD_SIDE_X: x / z = 1.15 times the Jacobian's clamp limit 1.3 (W/2)/fx, so J uses the
      clamped x, yet its 3-sigma footprint reaches into the image from the right;
    - FD_SIDE_Y: the same below the image, for the y clamp;
    - FD_OPAQUE: logit 9 (o = 0.99988) and about 8 px across, behind the others, so alpha
      = min(0.99, o e^power) is held at 0.99 on the pixels within about 1 px of its centre;
    - FD_DARK: a red SH sum near -0.4, so its red colour is clamped at 0 (degree 3: with
      higher-order red terms, whose gradient and direction terms the clamp removes)."""
    rng = np.random.default_rng(seed)
    cam = I.pinhole(40, 36, 60.0, (0.3, -0.2, -2.2), (0.0, 0.0, 0.0), 0.01)
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    limx = 1.3 * (0.5 * cam.width) / cam.fx
    limy = 1.3 * (0.5 * cam.height) / cam.fy
    cam_means = np.array([[1.15 * limx * 2.0, 0.1, 2.0],
                          [0.1, 1.15 * limy * 2.0, 2.0],
                          [0.25, -0.2, 3.2],
                          [-0.45, -0.35, 2.1]])
    special = (cam_means - t) @ R  # world = R^T (c - t)
    nc = I.n_sh_coeffs(deg)
    n = 24
    means = np.concatenate([special, rng.uniform(-0.5, 0.5, (n, 3))])
    log_scales = np.concatenate([np.log([[0.35] * 3, [0.35] * 3, [0.45] * 3, [0.12] * 3]),
                                 rng.normal(-2.6, 0.3, (n, 3))])
    logits = np.concatenate([[0.5, 0.5, 9.0, 1.0], rng.normal(0.0, 1.0, n)])
    rgb = np.concatenate([[[0.7, 0.5, 0.3], [0.3, 0.6, 0.8], [0.8, 0.7, 0.2], [-0.4, 0.6, 0.4]],
                          rng.uniform(0.2, 0.8, (n, 3))])
    sh = np.zeros((n + 4, nc, 3), np.float32)
    sh[:, 0, :] = (rgb - 0.5) / Y00
    if deg:
        sh[:, 1:, :] = rng.normal(0, 0.2, (n + 4, nc - 1, 3))
        sh[FD_DARK, 1:, 0] = rng.normal(0, 0.05, nc - 1)
    sc = _scene(means, log_scales, rng.standard_normal((n + 4, 4)), logits, sh=sh, deg=deg)
    return sc, cam


def _fd_check(deg, seed=20):
    """Central finite differences (h = 1e-7 max(1, |p|)) of L = sum wC * image + sum wT * T
    against the oracle's backward, for 40 seeded parameters of every array and for every
    parameter of the four clamp Gaussians, leaving out parameters whose +-h changes a
    discrete decision (visibility, rectangle, contributors, subset order, clamp branches).
    Returns the number of parameters checked and the clamp Gaussians' checked count."""
    sc, cam = _fd_scene(deg, seed + deg)
    rng = np.random.default_rng(seed + 100 + deg)
    perm, off, _ = I.kd_partition(sc.means, 2)
    inv = np.argsort(perm)
    specials = inv[:4]  # positions of the clamp Gaussians after the partition's reordering
    sc = sc.take(perm)
    o = O.opts(eps_T=1e-4, eps_comp=1e-4)
    flags, ncl = O.branch_stats(sc, off, cam, o)
    vis, _, _ = O.bin(sc, cam)
    assert vis[specials].all()
    assert flags[specials[FD_SIDE_X]] & 1, "x clamp of the Jacobian not reached"
    assert flags[specials[FD_SIDE_Y]] & 2, "y clamp of the Jacobian not reached"
    assert ncl[specials[FD_OPAQUE]] > 0, "alpha clamp not reached"
    assert flags[specials[FD_DARK]] & 4, "colour clamp not reached"
    wC = rng.standard_normal((3, cam.height, cam.width))
    wT = rng.standard_normal((cam.height, cam.width))
    grads = O.backward_view(sc, off, cam, wC, wT, o)
    for g in specials:  # each clamp Gaussian takes part in the image
        assert np.abs(grads[0][g]).max() > 0.0
    base_sig = _signature(sc, off, cam, o)
    arrays = list(sc.arrays())
    checked = checked_special = 0
    for ai, (arr, g) in enumerate(zip(arrays, grads)):
        per = arr.size // sc.n
        flat = arr.reshape(-1)
        gflat = g.reshape(-1)
        idx = set(rng.choice(flat.size, size=min(flat.size, 40), replace=False).tolist())
        sp = {int(s) * per + k for s in specials for k in range(per)}
        for j in sorted(idx | sp):
            x0 = float(flat[j])
            h = 1e-7 * max(1.0, abs(x0))
            vals = []
            ok = True
            for sgn in (1, -1):
                sc2 = I.Scene(*[a.astype(np.float64).copy() for a in arrays], sc.sh_degree)
                sc2.arrays()[ai].reshape(-1)[j] = x0 + sgn * h
                if _signature(sc2, off, cam, o) != base_sig:
                    ok = False
                    break
                vals.append(_loss(sc2, off, cam, o, wC, wT))
            if not ok:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            scale = max(1e-3, np.abs(gflat).max() * 1e-3)
            assert abs(fd - gflat[j]) <= 1e-4 * max(abs(fd), scale), (ai, j, fd, gflat[j])
            checked += 1
            checked_special += j in sp
    return checked, checked_special, sum(len(range(a.size // sc.n)) for a in arrays) * 4


@pytest.mark.parametrize("deg", [0, 3])
def test_backward_matches_central_finite_differences(deg):
    checked, checked_special, n_special = _fd_check(deg)
    assert checked >= 150
    assert checked_special >= 0.8 * n_special


# --------------------------------------------------------------------------- Adam
def test_adam_matches_torch_optim_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    p0 = rng.standard_normal(1000)
    p = p0.copy(); m = np.zeros_like(p); v = np.zeros_like(p)
    tp = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 6):
        g = rng.standard_normal(1000)
        O.adam(p, g, m, v, 1e-2, 0.9, 0.999, 1e-15, step)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------- regression
def test_oracle_regression_fixture():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_regression_small.json")
    with open(path) as f:
        g = json.load(f)
    arr = g["inputs"]
    sc = I.Scene(*(np.asarray(arr[k], np.float32) for k in
                   ("means", "log_scales", "quats", "opacity_logits", "sh")), g["sh_degree"])
    c = g["camera"]
    cam = I.Camera(np.asarray(c["R"], np.float32), np.asarray(c["t"], np.float32), c["fx"],
                   c["fy"], c["cx"], c["cy"], c["width"], c["height"], c["near"])
    o = O.opts(tile=8)
    view = O.render_view(sc, np.asarray(g["offsets"]), cam, o)
    np.testing.assert_allclose(view["image"], np.asarray(g["image"]), atol=1e-12)
    np.testing.assert_allclose(view["T"], np.asarray(g["T"]), atol=1e-12)
    gr = O.backward_view(sc, np.asarray(g["offsets"]), cam, np.ones((3, cam.height, cam.width)),
                         None, o)
    np.testing.assert_allclose(gr[0], np.asarray(g["grad_means"]), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(gr[3], np.asarray(g["grad_opacity_logits"]), rtol=1e-9, atol=1e-12)


# --------------------------------------------------------------------------- saturation skipping
def test_cell_order_is_a_visibility_order():
    # for every ordered pair (i before j) some axis-aligned plane separates the two cells
    # with the eye not strictly on j's side (what a BSP's front-to-back order guarantees);
    # the product's implementation gives the same order
    from paper_2606_18588_gb300 import visibility as Vz
    rng = np.random.default_rng(5)
    for K in (2, 4, 8, 16):
        means = rng.normal(0.0, 3.0, (4000, 3))
        _, _, boxes = I.kd_partition(means.astype(np.float32), K)
        for _ in range(12):
            eye = rng.uniform(-12.0, 12.0, 3)
            order = O.cell_order(boxes, eye)
            assert sorted(order) == list(range(K))
            assert order == Vz.front_to_back(boxes, eye)
            for a in range(K):
                for c in range(a + 1, K):
                    i, j = order[a], order[c]
                    lo_i, hi_i, lo_j, hi_j = boxes[i, 0], boxes[i, 1], boxes[j, 0], boxes[j, 1]
                    ok = any((hi_i[x] <= lo_j[x] and eye[x] <= lo_j[x]) or
                             (lo_i[x] >= hi_j[x] and eye[x] >= hi_j[x]) for x in range(3))
                    assert ok, (K, eye, order, i, j)


def _saturating_slabs(seed, half_middle=False):
    """Three dense opaque slabs one behind the other (camera at z = -3 looking along +z),
    and the three cells split at z = -0.4 and z = 0.4.  half_middle: the middle slab
    ends at x = 0.1, so the pixels saturated after two slabs end inside a column of tiles."""
    rng = np.random.default_rng(seed)
    per = (4000, 4000, 4000)
    means, ls, logits = [], [], []
    for k, n in enumerate(per):
        m = rng.uniform(-1.8, 1.8, (n, 3))
        if half_middle and k == 1:
            m[:, 0] = rng.uniform(-1.8, 0.1, n)
        m[:, 2] = -0.8 + 0.8 * k + rng.uniform(-0.15, 0.15, n)
        means.append(m)
        ls.append(rng.normal(-2.6, 0.15, (n, 3)))
        logits.append(rng.normal(4.0, 0.5, n))
    n = sum(per)
    sc = _scene(np.concatenate(means), np.concatenate(ls), rng.standard_normal((n, 4)),
                np.concatenate(logits), rgb=rng.uniform(0, 1, (n, 3)))
    offsets = np.concatenate([[0], np.cumsum(per)])
    inf = np.inf
    boxes = np.array([[[-inf, -inf, -inf], [inf, inf, -0.4]],
                      [[-inf, -inf, -0.4], [inf, inf, 0.4]],
                      [[-inf, -inf, 0.4], [inf, inf, inf]]])
    return sc, offsets, boxes


def test_saturation_skipping_leaves_the_image_and_gradients_unchanged():
    # subsets rendered front to back; a later subset leaves a pixel empty where the prefix
    # transmittance is below eps_comp, and a tile not rendered at all when that holds at
    # all its pixels.  The composite skips such subsets per pixel anyway, so on a
    # depth-separated scene images and gradients are exactly those of the full render
    sc, off, boxes = _saturating_slabs(21)
    cam = _cam(64, 48)
    order = O.cell_order(boxes, cam.eye)
    assert order == [0, 1, 2]
    o = O.opts()
    full = O.render_view(sc, off, cam, o)
    skipr = O.render_view(sc, off, cam, o, order=order)
    B = 16
    tw, th = (cam.width + B - 1) // B, (cam.height + B - 1) // B
    assert skipr["skip"][0].sum() == 0 and skipr["skip"][2].sum() > 0
    # every skip decision follows from the prefix of the returned partials
    prefix = np.ones((cam.height, cam.width))
    for r, m in enumerate(order):
        pad = np.zeros((th * B, tw * B))
        pad[:cam.height, :cam.width] = prefix
        tmax = pad.reshape(th, B, tw, B).max(axis=(1, 3)).reshape(-1)
        expect = (tmax < o.eps_comp) if r > 0 else np.zeros(tw * th, bool)
        assert np.array_equal(skipr["skip"][m].astype(bool), expect)
        prefix = prefix * skipr["Tp"][m]
    np.testing.assert_allclose(skipr["image"], full["image"], atol=1e-12, rtol=0)
    np.testing.assert_allclose(skipr["T"], full["T"], atol=1e-12, rtol=0)
    rng = np.random.default_rng(2)
    dC = rng.standard_normal((3, cam.height, cam.width))
    g_full = O.backward_view(sc, off, cam, dC, None, o)
    g_skip = O.backward_view(sc, off, cam, dC, None, o, order=order)
    for a, b in zip(g_full, g_skip):
        np.testing.assert_allclose(b, a, atol=1e-12, rtol=1e-10)


def test_saturation_skipping_empties_exactly_the_saturated_pixels():
    # Sec. 4.2: saturated pixels leave a later subset's pixel set.  Where the prefix of the
    # subsets rendered before is below eps_comp the partial is empty (C = 0, T = 1, D = 0);
    # everywhere else it is the partial of the render without skipping, also on the open
    # pixels of tiles that are partly saturated (a tile-only skip would fail the first
    # check there, a skip of open pixels the second)
    sc, off, boxes = _saturating_slabs(23, half_middle=True)
    cam = _cam(64, 48)
    order = O.cell_order(boxes, cam.eye)
    o = O.opts()
    full = O.render_view(sc, off, cam, o)
    skipr = O.render_view(sc, off, cam, o, order=order)
    B = 16
    tw, th = (cam.width + B - 1) // B, (cam.height + B - 1) // B
    prefix = np.ones((cam.height, cam.width))
    partial_tiles = 0
    for r, m in enumerate(order):
        if r > 0:
            shut = prefix < o.eps_comp  # the same FP64 products as the oracle's, same order
            assert np.all(skipr["Cp"][m][:, shut] == 0.0)
            assert np.all(skipr["Tp"][m][shut] == 1.0) and np.all(skipr["Dp"][m][shut] == 0.0)
            np.testing.assert_array_equal(skipr["Cp"][m][:, ~shut], full["Cp"][m][:, ~shut])
            np.testing.assert_array_equal(skipr["Tp"][m][~shut], full["Tp"][m][~shut])
            np.testing.assert_array_equal(skipr["Dp"][m][~shut], full["Dp"][m][~shut])
            pad = np.zeros((th * B, tw * B), bool)
            pad[:cam.height, :cam.width] = shut
            per_tile = pad.reshape(th, B, tw, B).sum(axis=(1, 3)).reshape(-1)
            n_in = np.zeros((th * B, tw * B), int)
            n_in[:cam.height, :cam.width] = 1
            n_in = n_in.reshape(th, B, tw, B).sum(axis=(1, 3)).reshape(-1)
            partial_tiles += int(((per_tile > 0) & (per_tile < n_in)).sum())
        prefix = prefix * skipr["Tp"][m]
    assert partial_tiles > 0


def test_saturation_skipping_drops_a_front_subset_when_ordered_wrongly():
    # the skip is only as good as the order: rendering back to front skips tiles of the
    # front slab and changes the image (the pins above are not vacuous)
    sc, off, boxes = _saturating_slabs(22)
    cam = _cam(64, 48)
    o = O.opts()
    full = O.render_view(sc, off, cam, o)
    wrong = O.render_view(sc, off, cam, o, order=[2, 1, 0])
    assert wrong["skip"][0].sum() > 0
    assert np.abs(wrong["image"] - full["image"]).max() > 1e-2


def _prefix_state(Tp, order, eps, lim=None):
    """Brute force of the re-evaluated saturation state from the partial transmittances:
    r + 1 for the first rank r (below lim) whose prefix product is below eps, else 255
    (also when r + 1 = K)."""
    K, H, W = Tp.shape
    lim = np.full((H, W), K) if lim is None else np.minimum(lim.astype(int), K)
    out = np.full((H, W), 255, np.uint8)
    done = np.zeros((H, W), bool)
    prefix = np.ones((H, W))
    for r, m in enumerate(order):
        prefix = prefix * Tp[m]
        hit = ~done & (r < lim) & (prefix < eps)
        out[hit] = r + 1 if r + 1 < K else 255
        done |= hit
    return out


def test_stale_state_prunes_exactly_the_ranks_it_names():
    # Sec. 4.2 step 2: with a view's stale state sat, the subset at rank r leaves pixel p
    # empty exactly when r >= sat[p]; every other pixel of every partial is the full
    # render's, and a tile with no open pixel is not rendered.  Random states, including
    # 0 (even the front subset pruned) and values >= K (nothing pruned)
    sc, off, boxes = _saturating_slabs(24, half_middle=True)
    cam = _cam(64, 48)
    order = O.cell_order(boxes, cam.eye)
    o = O.opts()
    K = len(order)
    full = O.render_view(sc, off, cam, o)
    rng = np.random.default_rng(3)
    sat = rng.choice(np.array([0, 1, 2, 3, 200, 255], np.uint8), (cam.height, cam.width))
    sat[:16, :16] = 1  # one tile where only the front subset is open
    sat[16:32, 16:32] = 0  # one tile pruned from every subset
    st = O.render_view(sc, off, cam, o, order=order, sat=sat)
    B = 16
    tw, th = (cam.width + B - 1) // B, (cam.height + B - 1) // B
    for r, m in enumerate(order):
        shut = r >= sat
        assert np.all(st["Cp"][m][:, shut] == 0.0)
        assert np.all(st["Tp"][m][shut] == 1.0) and np.all(st["Dp"][m][shut] == 0.0)
        np.testing.assert_array_equal(st["Cp"][m][:, ~shut], full["Cp"][m][:, ~shut])
        np.testing.assert_array_equal(st["Tp"][m][~shut], full["Tp"][m][~shut])
        pad = np.ones((th * B, tw * B), bool)
        pad[:cam.height, :cam.width] = shut
        expect = pad.reshape(th, B, tw, B).all(axis=(1, 3)).reshape(-1)
        assert np.array_equal(st["skip"][m].astype(bool), expect)
    assert st["skip"][order[0]][tw + 1] == 1 and st["skip"][order[1]][0] == 1
    # the image is the composite of these partials; the re-evaluated state follows from
    # them, examining the ranks below min(sat, K) only
    np.testing.assert_array_equal(st["sat"], _prefix_state(st["Tp"], order, o.eps_comp, sat))
    assert K == 3


def test_stale_state_of_a_visit_reproduces_the_exact_skip_on_the_next():
    # a first visit prunes nothing (state 255) and renders the full image; its re-evaluated
    # state is the first saturated rank of each pixel (brute force from its partials).  The
    # next visit with that state renders exactly the partials, skip flags, image and
    # gradients of the exact (same-visit) saturation skip, and re-evaluates to the same state
    sc, off, boxes = _saturating_slabs(25, half_middle=True)
    cam = _cam(64, 48)
    order = O.cell_order(boxes, cam.eye)
    o = O.opts()
    none = np.full((cam.height, cam.width), 255, np.uint8)
    full = O.render_view(sc, off, cam, o)
    v1 = O.render_view(sc, off, cam, o, order=order, sat=none)
    for key in ("image", "T", "Cp", "Tp", "Dp"):
        np.testing.assert_array_equal(v1[key], full[key])
    assert v1["skip"].sum() == 0
    s1 = v1["sat"]
    np.testing.assert_array_equal(s1, _prefix_state(v1["Tp"], order, o.eps_comp))
    assert (s1 == 2).sum() > 0 and (s1 == 255).sum() > 0  # pruned after two slabs, and open
    exact = O.render_view(sc, off, cam, o, order=order)
    v2 = O.render_view(sc, off, cam, o, order=order, sat=s1)
    for key in ("image", "T", "Cp", "Tp", "Dp", "skip"):
        np.testing.assert_array_equal(v2[key], exact[key])
    np.testing.assert_array_equal(v2["sat"], s1)
    rng = np.random.default_rng(4)
    dC = rng.standard_normal((3, cam.height, cam.width))
    g_exact = O.backward_view(sc, off, cam, dC, None, o, order=order)
    g_stale = O.backward_view(sc, off, cam, dC, None, o, order=order, sat=s1)
    for a, b in zip(g_exact, g_stale):  # (the oracle adds 2-D gradients in thread order)
        np.testing.assert_allclose(b, a, atol=1e-12, rtol=1e-10)


def test_stale_state_brings_pruned_ranks_back_when_the_front_clears():
    # the front slab turns nearly transparent after the state was taken: the stale visit
    # still prunes the back slab (its image misses it: the cost of a stale state), its
    # re-evaluation finds the prefix above eps_comp up to the old state and brings every
    # pruned rank back, and the visit after that renders the full image again
    sc, off, boxes = _saturating_slabs(26)
    cam = _cam(64, 48)
    order = O.cell_order(boxes, cam.eye)
    o = O.opts()
    none = np.full((cam.height, cam.width), 255, np.uint8)
    s1 = O.render_view(sc, off, cam, o, order=order, sat=none)["sat"]
    assert (s1 < 255).sum() > 0
    logits = sc.opacity_logits.copy()
    logits[: off[2]] = -6.0  # the front and middle slabs nearly transparent
    sc2 = I.Scene(sc.means, sc.log_scales, sc.quats, logits, sc.sh, sc.sh_degree)
    full2 = O.render_view(sc2, off, cam, o)
    v2 = O.render_view(sc2, off, cam, o, order=order, sat=s1)
    back = s1 <= 2  # pixels where the back slab was pruned
    assert np.abs(v2["image"] - full2["image"]).max(axis=0)[back].max() > 1e-2
    np.testing.assert_array_equal(v2["sat"], _prefix_state(v2["Tp"], order, o.eps_comp, s1))
    assert np.all(v2["sat"][back] == 255)
    v3 = O.render_view(sc2, off, cam, o, order=order, sat=v2["sat"])
    np.testing.assert_allclose(v3["image"], full2["image"], atol=1e-12, rtol=0)


# --------------------------------------------------------------------------- D-SSIM loss
def test_ssim_window_sum_is_the_windowed_sum():
    # brute force: every output pixel sums the 11 x 11 window of weights w_i w_j over the
    # pixels inside the image
    rng = np.random.default_rng(1)
    a = rng.uniform(0, 1, (9, 13))
    w = O.ssim_window()
    assert abs(w.sum() - 1.0) < 1e-15 and np.allclose(w, w[::-1])
    assert np.isclose(w[5] / w[4], np.exp(0.5 / 1.5 ** 2))  # Gaussian, sigma 1.5
    ref = np.zeros_like(a)
    for y in range(9):
        for x in range(13):
            for i in range(11):
                for j in range(11):
                    yy, xx = y + i - 5, x + j - 5
                    if 0 <= yy < 9 and 0 <= xx < 13:
                        ref[y, x] += w[i] * w[j] * a[yy, xx]
    np.testing.assert_allclose(O._window_sum(a, w), ref, rtol=1e-13, atol=1e-15)


def test_ssim_closed_forms():
    # identical images: SSIM = 1, loss 0, zero gradient
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (3, 20, 24))
    loss, g = O.loss_l1_dssim([x], [x])
    assert abs(loss) < 1e-12 and np.abs(g[0]).max() < 1e-12
    # constant images a, b: away from the border every window sees only a and b, the
    # variances vanish, and S = (2ab + C1) / (a^2 + b^2 + C1)
    a, b = 0.3, 0.7
    S, _, _, _ = O.ssim_terms(np.full((30, 30), a), np.full((30, 30), b))
    expect = (2 * a * b + O.SSIM_C1) / (a * a + b * b + O.SSIM_C1)
    np.testing.assert_allclose(S[5:-5, 5:-5], expect, rtol=1e-12)
    # lam = 0 is the plain L1 loss
    y = rng.uniform(0, 1, x.shape)
    loss0, g0 = O.loss_l1_dssim([x], [y], lam=0.0)
    assert np.isclose(loss0, np.abs(x - y).mean())
    np.testing.assert_allclose(g0[0], np.sign(x - y) / x.size)


def test_ssim_gradient_finite_differences():
    rng = np.random.default_rng(3)
    xs = [rng.uniform(0.1, 0.9, (3, 14, 17)), rng.uniform(0.1, 0.9, (3, 9, 11))]
    ys = [rng.uniform(0, 1, a.shape) for a in xs]
    _, g = O.loss_l1_dssim(xs, ys, lam=0.2)
    h = 1e-6
    for v, idx in [(0, (0, 0, 0)), (0, (1, 7, 8)), (0, (2, 13, 16)), (1, (1, 0, 10)), (1, (0, 4, 5))]:
        xp = [a.copy() for a in xs]
        xm = [a.copy() for a in xs]
        xp[v][idx] += h
        xm[v][idx] -= h
        fd = (O.loss_l1_dssim(xp, ys)[0] - O.loss_l1_dssim(xm, ys)[0]) / (2 * h)
        assert abs(fd - g[v][idx]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (v, idx, fd, g[v][idx])


# --------------------------------------------------------------------------- cross-boundary
# Per-ray filtering of cross-boundary Gaussians (Sec. 8.1): the configuration of the
# paper's example.  Two cells split at x = 0; G1 (depth 2) and G3 (depth 4) belong to cell
# 0, G2 (depth 3) and G4 (depth 5) to cell 1; G3's 3-sigma support reaches into cell 1.
_INF = float("inf")
_TWO_CELLS = np.array([[[-_INF, -_INF, -_INF], [0.0, _INF, _INF]],
                       [[0.0, -_INF, -_INF], [_INF, _INF, _INF]]])


def _cross_example(with_g3=True):
    # camera at z = -1 looking along +z: depth = z + 1
    g = [((-0.2, 0.0, 1.0), math.log(0.05), (1.0, 0.2, 0.2)),   # G1, cell 0
         ((-0.02, 0.0, 3.0), math.log(0.3), (0.2, 1.0, 0.2)),   # G3, cell 0, crosses x = 0
         ((0.2, 0.0, 2.0), math.log(0.02), (0.2, 0.2, 1.0)),    # G2, cell 1
         ((0.3, 0.0, 4.0), math.log(0.03), (0.9, 0.9, 0.1))]    # G4, cell 1
    if not with_g3:
        g = [g[0], g[2], g[3]]
    n = len(g)
    sc = _scene([x[0] for x in g], [[x[1]] * 3 for x in g], [[1.0, 0.0, 0.0, 0.0]] * n,
                [_logit(0.8)] * n, rgb=[x[2] for x in g])
    off = np.array([0, n - 2, n])
    cam = I.pinhole(64, 64, 60.0, (0.0, 0.0, -1.0), (0.0, 0.0, 1.0), 0.01)
    return sc, off, cam


def test_cross_boundary_filter_removes_g3_only_where_both_cells_are_seen():
    o = O.opts(eps_T=0.0, eps_comp=0.0)
    sc, off, cam = _cross_example()
    sc3, off3, _ = _cross_example(with_g3=False)
    filt = O.render_view(sc, off, cam, o, cells=_TWO_CELLS)["image"]
    full = O.render_view(sc, off, cam, o)["image"]
    without = O.render_view(sc3, off3, cam, o)["image"]
    # Omega of cell 1: the bounding rectangle of the tile rectangles of its paired Gaussians
    B, tw = 16, 4
    c1 = sc.subset(2, 4)
    start, lst = O.tile_lists(c1, cam)
    _, rect, _ = O.bin(c1, cam)
    r = rect[np.unique(lst)] // B
    omega1 = [ty * tw + tx for ty in range(r[:, 2].min(), r[:, 3].max() + 1)
              for tx in range(r[:, 0].min(), r[:, 1].max() + 1)]
    start3, _ = O.tile_lists(sc.subset(1, 2), cam)
    g3_tiles = np.nonzero(np.diff(start3) > 0)[0]
    assert set(omega1) < set(g3_tiles)  # G3 also covers tiles cell 1 does not see
    changed = 0
    for t in range(16):
        ys, xs = slice((t // tw) * B, (t // tw + 1) * B), slice((t % tw) * B, (t % tw + 1) * B)
        ref = without if t in omega1 else full
        assert np.array_equal(filt[:, ys, xs], ref[:, ys, xs]), t
        changed += int(not np.array_equal(full[:, ys, xs], without[:, ys, xs]))
    assert changed >= 3  # G3 matters on its tiles, so both branches are exercised


def test_cross_boundary_filter_keeps_gaussians_outside_the_depth_overlap():
    # G3 moved in front of cell 1's depth range: kept everywhere
    o = O.opts(eps_T=0.0, eps_comp=0.0)
    sc, off, cam = _cross_example()
    sc.means[1, 2] = 1.5  # depth 2.5 < D_1 = [3, 5]
    filt = O.render_view(sc, off, cam, o, cells=_TWO_CELLS)["image"]
    full = O.render_view(sc, off, cam, o)["image"]
    assert np.array_equal(filt, full)


def test_cross_boundary_filter_is_the_identity_without_crossing_gaussians():
    rng = np.random.default_rng(8)
    sc = I.uniform_scene(6000, 8, 1, log_scale_mu=-6.0, log_scale_sigma=0.2)
    perm, off, boxes = I.kd_partition(sc.means, 4)
    sc = sc.take(perm)
    planes = [boxes[k, s, a] for k in range(4) for s in range(2) for a in range(3)
              if np.isfinite(boxes[k, s, a])]
    far = np.all([np.abs(sc.means[:, a] - p) > 0.05 for p in set(planes) for a in range(3)],
                 axis=0)
    keep = np.nonzero(far)[0]
    cell = np.searchsorted(off, keep, side="right") - 1
    sc = sc.take(keep)
    off = np.concatenate([[0], np.cumsum(np.bincount(cell, minlength=4))])
    cam = _cam(96, 80)
    o = O.opts()
    a = O.render_view(sc, off, cam, o, cells=boxes)
    b = O.render_view(sc, off, cam, o)
    assert np.array_equal(a["image"], b["image"])
    dC = rng.standard_normal((3, 80, 96))
    ga = O.backward_view(sc, off, cam, dC, None, o, cells=boxes)
    gb = O.backward_view(sc, off, cam, dC, None, o)
    # the oracle's threads add per-Gaussian sums in any order: equal up to rounding
    assert all(np.allclose(x, y, rtol=1e-12, atol=1e-15) for x, y in zip(ga, gb))


# --------------------------------------------------------------------------- flip bounds
@pytest.mark.parametrize("skipping", [False, True])
def test_flip_bounds_cover_every_flipped_decision(skipping):
    """The oracle's flip bound of an ambiguous pixel covers the result of taking its flagged
    decisions the other way.  Moving alpha_min, eps_T and eps_comp by 0.9 of their relative
    margins flips exactly decisions that the oracle flags (and whatever later stops those
    flips move); every pixel must then stay within its bound of the unmoved render, and an
    unflagged pixel must not change at all."""
    sc = I.cluster_scene(20_000, 2, 3)
    cam = I.orbit_cameras(1, 3, [(333, 197)])[0]
    perm, off, boxes = I.kd_partition(sc.means, 4)
    sc = sc.take(perm)
    order = O.cell_order(boxes, cam.eye) if skipping else None
    base_o = O.opts()
    base = O.render_view(sc, off, cam, base_o, order=order, bounds=True)
    amb = base["amb"] != 0
    assert 0 < amb.mean() < 0.01
    fb = base["flip"]
    moved_any = False
    for sa, st, sc_ in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                        (1, -1, 1), (-1, 1, -1)]:
        o = O.opts(alpha_min=base_o.alpha_min * (1 + 0.9 * sa * base_o.amb_alpha),
                   eps_T=base_o.eps_T * (1 + 0.9 * st * base_o.amb_T),
                   eps_comp=base_o.eps_comp * (1 + 0.9 * sc_ * base_o.amb_T))
        r = O.render_view(sc, off, cam, o, order=order)
        d_img = np.abs(r["image"] - base["image"]).max(axis=0)
        d_T = np.abs(r["T"] - base["T"])
        assert d_img[~amb].max(initial=0.0) == 0.0 and d_T[~amb].max(initial=0.0) == 0.0
        assert (d_img <= fb["image"] * (1 + 1e-9) + 1e-15).all()
        assert (d_T <= fb["T"] * (1 + 1e-9) + 1e-15).all()
        for m in range(len(off) - 1):
            dC = np.abs(r["Cp"][m] - base["Cp"][m]).max(axis=0)
            assert (dC <= fb["partC"][m] * (1 + 1e-9) + 1e-15).all()
            assert (np.abs(r["Tp"][m] - base["Tp"][m]) <= fb["partT"][m] * (1 + 1e-9) + 1e-15).all()
            assert (np.abs(r["Dp"][m] - base["Dp"][m]) <= fb["partD"][m] * (1 + 1e-9) + 1e-15).all()
        moved_any |= bool(d_img.max() > 0)
    assert moved_any


def test_composite_flip_bound_covers_a_swapped_near_tie():
    """Two partials whose normalised depths differ by less than the key margin: the oracle
    flags the pixel, and its bound covers compositing them the other way round (Eq. 5 with
    the pair's order exchanged)."""
    rng = np.random.default_rng(8)
    K, H, W = 3, 4, 5
    Tp = rng.uniform(0.2, 0.9, (K, H, W))
    Cp = rng.uniform(0, 1, (K, 3, H, W)) * (1 - Tp)[:, None]
    z = rng.uniform(1, 10, (K, H, W))
    z[1] = z[0] * (1 + 3e-6)            # near-tied with subset 0 everywhere
    Dp = z * (1 - Tp)
    o = O.opts(eps_comp=0.0)
    base = O.composite(Cp, Tp, Dp, o, bounds=True)
    assert (base["amb"] != 0).all()
    z2 = z.copy()
    z2[1] = z[0] * (1 - 3e-6)           # the pair the other way round
    swapped = O.composite(Cp, Tp, z2 * (1 - Tp), o)
    d = np.abs(swapped["image"] - base["image"]).max(axis=0)
    assert d.max() > 1e-3
    assert (d <= base["flip"]["image"] * (1 + 1e-9) + 1e-15).all()
