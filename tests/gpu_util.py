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
