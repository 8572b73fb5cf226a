"""Helpers for the GPU tests: move a seeded scene to the device and drive the C ABI."""
import numpy as np
import torch

from paper_2606_18588_gb300 import splx as S

PIXEL_TOL = 1e-4      # max-abs on [0,1] pixels outside the ambiguity guard band
GRAD_TOL = 1e-3       # relative L2 per parameter group


def to_device(scene):
    return {k: torch.from_numpy(np.ascontiguousarray(a)).cuda() for k, a in
            zip(("means", "log_scales", "quats", "opacity_logits", "sh"), scene.arrays())}


def subset_struct(dev, lo, hi, deg):
    return S.gaussians(dev["means"][lo:hi], dev["log_scales"][lo:hi], dev["quats"][lo:hi],
                       dev["opacity_logits"][lo:hi], dev["sh"][lo:hi], deg)


def zeros_like_params(dev):
    return {k: torch.zeros_like(v) for k, v in dev.items()}


def params_struct(d, lo, hi, deg):
    return S.params(d["means"][lo:hi], d["log_scales"][lo:hi], d["quats"][lo:hi],
                    d["opacity_logits"][lo:hi], d["sh"][lo:hi], deg)


def render_view(ctx, dev, offsets, cam, o, deg, keep_state=True):
    """K local renders + composite through the C ABI.  Returns (image, T, parts, states)."""
    K = len(offsets) - 1
    parts, states = [], []
    for k in range(K):
        p = S.new_partial(cam.height, cam.width)
        st = S.render_partial(ctx, subset_struct(dev, int(offsets[k]), int(offsets[k + 1]), deg),
                              cam, o, p, keep_state=keep_state)
        parts.append(p)
        states.append(st)
    img = torch.empty(3, cam.height, cam.width, device="cuda")
    T = torch.empty(cam.height, cam.width, device="cuda")
    S.composite(ctx, parts, cam.width, cam.height, o, img, T)
    torch.cuda.synchronize()
    return img, T, parts, states


def backward_view(ctx, dev, offsets, cam, o, deg, parts, states, dLdC, dLdT=None):
    K = len(offsets) - 1
    g = zeros_like_params(dev)
    subs = [subset_struct(dev, int(offsets[k]), int(offsets[k + 1]), deg) for k in range(K)]
    grads = [params_struct(g, int(offsets[k]), int(offsets[k + 1]), deg) for k in range(K)]
    S.backward(ctx, subs, cam, parts, states, dLdC, dLdT, o, grads)
    torch.cuda.synchronize()
    return g


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))


def decode_records(rec):
    """(visible, rect[n,4], depth_bits) from exported 64-byte records."""
    rx = rec[:, 7].view(np.uint32)
    ry = rec[:, 11].view(np.uint32)
    x0, x1 = (rx & 0xFFFF).astype(np.int32), (rx >> 16).astype(np.int32)
    y0, y1 = (ry & 0xFFFF).astype(np.int32), (ry >> 16).astype(np.int32)
    vis = (x0 <= x1).astype(np.int32)
    rect = np.stack([x0, x1, y0, y1], axis=1)
    depth_bits = rec[:, 6].view(np.uint32)
    return vis, rect, depth_bits


# The oracle flags a pixel ambiguous when one of its discrete decisions (alpha >= alpha_min,
# power <= 0, the transmittance stop, the saturation cut, the order of near-tied subset
# keys) lies within FP32's reach of its threshold, so that an FP32 kernel may take either
# side.  Such pixels are not skipped: each is checked against the oracle's flip bound, how
# far taking those decisions the other way can move it (blend_pixel / composite_bounds in
# the oracle, pinned by tests/test_oracle_pins.py).  BAND_BUDGET caps the share of a test's
# pixels checked that way; at about 2.4e-5 per alpha evaluation near the threshold and
# 1e-3 per pixel that stops on eps_T, the workloads here stay well inside it.
BAND_BUDGET = 0.01


def check_band(gpu, ref, amb, bound, tol=PIXEL_TOL, budget=BAND_BUDGET, label="", where=None):
    """One output plane ([H, W] or [C, H, W]) of the GPU against the oracle's: |gpu - ref| <=
    tol on every pixel outside the ambiguity band, and <= tol + the oracle's flip bound on
    every pixel inside it; the band may hold at most `budget` of the compared pixels
    (`where`, default all).  `tol` may be an array (broadcast to [H, W]).  Prints the band's
    share; returns (largest error outside the band, band share)."""
    err = np.abs(np.asarray(gpu, np.float64) - np.asarray(ref, np.float64))
    if err.ndim == 3:
        err = err.max(axis=0)
    sel = np.ones(err.shape, bool) if where is None else np.asarray(where, bool)
    band = (np.asarray(amb) != 0) & sel
    off = sel & ~band
    tol = np.broadcast_to(np.asarray(tol, np.float64), err.shape)
    bound = np.broadcast_to(np.asarray(bound, np.float64), err.shape)
    frac = float(band.sum()) / max(int(sel.sum()), 1)
    e_off = float(err[off].max(initial=0.0))
    print(f"[band] {label}: {int(band.sum())} of {int(sel.sum())} pixels in the ambiguity band "
          f"({frac:.2e}, budget {budget:g}); max error outside {e_off:.2e}, inside "
          f"{float(err[band].max(initial=0.0)):.2e} (largest bound "
          f"{float(bound[band].max(initial=0.0)):.2e})")
    bad_off = off & (err > tol)
    assert not bad_off.any(), f"{label}: {int(bad_off.sum())} pixels off the band beyond tolerance"
    bad_in = band & (err > tol + bound)
    assert not bad_in.any(), (f"{label}: {int(bad_in.sum())} band pixels beyond their flip bound, "
                              f"worst excess {float((err - tol - bound)[bad_in].max()):.3e}")
    assert frac <= budget, f"{label}: ambiguity band {frac:.2e} above its budget {budget:g}"
    return e_off, frac


def band_share(amb, budget=BAND_BUDGET, label="", where=None):
    """Share of the ambiguity band among the pixels of a gradient test, whose loss gradient
    is zero on the band (a flipped decision changes which Gaussians a pixel reaches, so its
    gradient is not comparable); asserted against the budget and printed."""
    sel = np.ones(np.shape(amb), bool) if where is None else np.asarray(where, bool)
    band = (np.asarray(amb) != 0) & sel
    frac = float(band.sum()) / max(int(sel.sum()), 1)
    print(f"[band] {label}: {int(band.sum())} of {int(sel.sum())} pixels in the ambiguity band "
          f"({frac:.2e}, budget {budget:g}), loss gradient zero there")
    assert frac <= budget, f"{label}: ambiguity band {frac:.2e} above its budget {budget:g}"
    return frac
