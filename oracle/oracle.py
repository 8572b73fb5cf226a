"""ctypes wrapper of the FP64 CPU oracle (splx_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg.  The product path never imports this module.

Every function takes float64 copies of the parameters, so finite differences can
perturb them in FP64; the FP32 binning specification rounds them to float itself.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "splx_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-ffp-contract=off keeps the FP32 spec uncontracted)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("near_plane", C.c_float)]


class Opts(C.Structure):
    _fields_ = [("tile", C.c_int32), ("eps_T", C.c_double), ("eps_comp", C.c_double),
                ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("bg", C.c_double * 3),
                ("amb_alpha", C.c_double), ("amb_power", C.c_double), ("amb_T", C.c_double),
                ("amb_key", C.c_double)]


_dp = C.POINTER(C.c_double)


class Bounds(C.Structure):
    _fields_ = [("image", _dp), ("T", _dp), ("partC", _dp), ("partT", _dp),
                ("cmax", C.c_double), ("dmax", C.c_double)]


class Params(C.Structure):
    _fields_ = [("means", _dp), ("log_scales", _dp), ("quats", _dp), ("opacity_logits", _dp),
                ("sh", _dp), ("n", C.c_int64), ("sh_degree", C.c_int32)]


class Grads(C.Structure):
    _fields_ = [("means", _dp), ("log_scales", _dp), ("quats", _dp), ("opacity_logits", _dp),
                ("sh", _dp)]


def _bind(path):
    """Loads an oracle build and declares its entry points."""
    lib_ = C.CDLL(path)
    P = C.c_void_p
    _declare(lib_, P)
    return lib_


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


@contextlib.contextmanager
def using(path):
    """Runs the wrapper's functions on another build of the oracle (for instance one with a
    planted mistake, compiled by a test from a modified copy of the source) inside the
    `with` block."""
    global _lib
    other = _bind(path)
    with _lock:
        saved, _lib = _lib, other
    try:
        yield other
    finally:
        with _lock:
            _lib = saved


def compile_variant(src_text: str, out_path: str) -> str:
    """Compiles oracle source text (the committed source with a test's change) to out_path
    with the same flags as build()."""
    src = out_path + ".cpp"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-fno-fast-math", "-o", out_path, src], check=True)
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _declare(L, P):
    L.orc_exp_spec.restype = C.c_float
    L.orc_exp_spec.argtypes = [C.c_float]
    L.orc_exp_spec_n.argtypes = [P, P, C.c_int64]
    L.orc_log_spec_n.argtypes = [P, P, C.c_int64]
    L.orc_sh_basis.argtypes = [P, C.c_int64, P]
    L.orc_sh_basis_grad.argtypes = [P, C.c_int64, P]
    L.orc_bin.argtypes = [P, P, P, P, P]
    L.orc_tile_lists.restype = C.c_int64
    L.orc_tile_lists.argtypes = [P, P, C.c_int32, C.c_double, P, P, C.c_int64]
    L.orc_project.argtypes = [P, P, P]
    L.orc_render.argtypes = [P, P, P, P, P, P, P, P, P, P, P, P]
    L.orc_composite.argtypes = [C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, P, P, P, P,
                                P]
    L.orc_render_view.argtypes = [P, P, C.c_int32, P, P, P, P, P, P, P, P, P, P, P, P,
                                  P, P, P]
    L.orc_backward_view.argtypes = [P, P, C.c_int32, P, P, P, P, P, P, P, P]
    L.orc_render_view_pruned.argtypes = [P, P, C.c_int32, P, P, P, P, P, P, P, P, P, P, P, P,
                                         P, P, P, P, P]
    L.orc_backward_view_pruned.argtypes = [P, P, C.c_int32, P, P, P, P, P, P, P, P, P]
    L.orc_adam.argtypes = [C.c_int64, P, P, P, P, C.c_double, C.c_double, C.c_double,
                           C.c_double, C.c_int64]
    L.orc_num_threads.restype = C.c_int
    L.orc_branch_stats.argtypes = [P, P, C.c_int32, P, P, P, P]


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _Keep:
    """Holds float64 copies of a scene alive while C code reads them."""

    def __init__(self, scene):
        self.arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in scene.arrays()]
        m, ls, q, o, sh = self.arrs
        self.p = Params(m.ctypes.data_as(_dp), ls.ctypes.data_as(_dp), q.ctypes.data_as(_dp),
                        o.ctypes.data_as(_dp), sh.ctypes.data_as(_dp), m.shape[0], scene.sh_degree)


def camera(cam) -> Camera:
    c = Camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).reshape(-1)]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32).reshape(-1)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height, c.near_plane = cam.width, cam.height, cam.near
    return c


def opts(tile=16, eps_T=1e-4, eps_comp=1e-4, alpha_min=1.0 / 255.0, alpha_max=0.99,
         bg=(0.0, 0.0, 0.0), amb_alpha=2e-5, amb_power=1e-5, amb_T=3e-4, amb_key=1e-5) -> Opts:
    o = Opts()
    o.tile, o.eps_T, o.eps_comp, o.alpha_min, o.alpha_max = tile, eps_T, eps_comp, alpha_min, alpha_max
    o.bg[:] = list(bg)
    o.amb_alpha, o.amb_power, o.amb_T, o.amb_key = amb_alpha, amb_power, amb_T, amb_key
    return o


def exp_spec(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(x)
    lib().orc_exp_spec_n(_ptr(x), _ptr(y), x.size)
    return y


def log_spec(x: np.ndarray) -> np.ndarray:
    """FP32 natural logarithm of the binning specification (arguments >= 1)."""
    x = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(x)
    lib().orc_log_spec_n(_ptr(x), _ptr(y), x.size)
    return y


def sh_basis(dirs: np.ndarray, grad: bool = False) -> np.ndarray:
    d = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    if grad:
        out = np.empty((d.shape[0], 16, 3))
        lib().orc_sh_basis_grad(_ptr(d), d.shape[0], _ptr(out))
    else:
        out = np.empty((d.shape[0], 16))
        lib().orc_sh_basis(_ptr(d), d.shape[0], _ptr(out))
    return out


def bin(scene, cam):
    """FP32 binning spec: (visible[n], rect[n,4] x0,x1,y0,y1, depth_bits[n] uint32)."""
    k = _Keep(scene)
    n = scene.n
    vis = np.empty(n, np.int32)
    rect = np.empty((n, 4), np.int32)
    db = np.empty(n, np.uint32)
    c = camera(cam)
    lib().orc_bin(C.byref(k.p), C.byref(c), _ptr(vis), _ptr(rect), _ptr(db))
    return vis, rect, db


def tile_lists(scene, cam, tile=16, alpha_min=1.0 / 255.0):
    """Sorted per-tile Gaussian lists after tile culling: (tile_start[ntiles+1] int64,
    list[int32])."""
    k = _Keep(scene)
    c = camera(cam)
    nt = ((cam.width + tile - 1) // tile) * ((cam.height + tile - 1) // tile)
    start = np.empty(nt + 1, np.int64)
    total = lib().orc_tile_lists(C.byref(k.p), C.byref(c), tile, alpha_min, _ptr(start), None, 0)
    lst = np.empty(max(total, 1), np.int32)
    got = lib().orc_tile_lists(C.byref(k.p), C.byref(c), tile, alpha_min, _ptr(start), _ptr(lst),
                               lst.size)
    assert got == total
    return start, lst[:total]


def project(scene, cam) -> np.ndarray:
    """FP64 projection [n,12]: u, v, A, B, C, o, r, g, b, depth, a, c (0 for culled)."""
    k = _Keep(scene)
    out = np.empty((scene.n, 12))
    c = camera(cam)
    lib().orc_project(C.byref(k.p), C.byref(c), _ptr(out))
    return out


def _bounds(H, W, K, image=True):
    out = dict(partC=np.zeros((K, H, W)), partT=np.zeros((K, H, W)))
    if image:
        out.update(image=np.zeros((H, W)), T=np.zeros((H, W)))
    b = Bounds(*(out[k].ctypes.data_as(_dp) if k in out else None
                 for k in ("image", "T", "partC", "partT")), 0.0, 0.0)
    return b, out


def render(scene, cam, o: Opts | None = None, tile_mask=None, bounds=False):
    """Local render of one subset: dict of C[3,H,W], T, D, last, ncontrib, amb, evaluated.
    With bounds: also "flip", the flip bounds of the ambiguous pixels (|delta C| <=
    partC cmax, |delta D| <= partC dmax, |delta T| <= partT; see orc_bounds)."""
    o = o or opts()
    k = _Keep(scene)
    c = camera(cam)
    H, W = cam.height, cam.width
    Cc = np.zeros((3, H, W)); T = np.ones((H, W)); D = np.zeros((H, W))
    last = np.full((H, W), -1, np.int32); nc = np.zeros((H, W), np.int32)
    amb = np.zeros((H, W), np.uint8); st = np.zeros(1, np.int64)
    tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
    bd, bout = _bounds(H, W, 1, image=False) if bounds else (None, None)
    lib().orc_render(C.byref(k.p), C.byref(c), C.byref(o), _ptr(tm), _ptr(Cc), _ptr(T), _ptr(D),
                     _ptr(last), _ptr(nc), _ptr(amb), _ptr(st),
                     C.byref(bd) if bd is not None else None)
    out = dict(C=Cc, T=T, D=D, last=last, ncontrib=nc, amb=amb, evaluated=int(st[0]))
    if bounds:
        out["flip"] = dict(C=bout["partC"][0] * bd.cmax, T=bout["partT"][0],
                           D=bout["partC"][0] * bd.dmax, cmax=bd.cmax, dmax=bd.dmax)
    return out


def composite(Cp, Tp, Dp, o: Opts | None = None, bounds=False):
    """Eq. 5 over K partials (C[K,3,H,W], T[K,H,W], D[K,H,W]): image, T, nused, amb; with
    bounds also "flip" (image, T): the effect of the flagged near-tied keys and saturation
    cuts of these exact partials."""
    o = o or opts()
    Cp = np.ascontiguousarray(Cp, np.float64); Tp = np.ascontiguousarray(Tp, np.float64)
    Dp = np.ascontiguousarray(Dp, np.float64)
    K, _, H, W = Cp.shape
    out = np.empty((3, H, W)); To = np.empty((H, W)); nu = np.empty((H, W), np.int32)
    amb = np.zeros((H, W), np.uint8)
    bi = np.zeros((H, W)) if bounds else None
    bt = np.zeros((H, W)) if bounds else None
    lib().orc_composite(K, H, W, _ptr(Cp), _ptr(Tp), _ptr(Dp), C.byref(o), _ptr(out), _ptr(To),
                        _ptr(nu), _ptr(amb), _ptr(bi), _ptr(bt))
    res = dict(image=out, T=To, nused=nu, amb=amb)
    if bounds:
        res["flip"] = dict(image=bi, T=bt)
    return res


def _order(order, K):
    if order is None:
        return None
    a = np.ascontiguousarray(order, np.int32)
    if sorted(a.tolist()) != list(range(K)):
        raise ValueError("order must be a permutation of the K subsets")
    return a


def _cells(cells, K):
    """[K, 2, 3] k-d boxes (lo, hi; infinite on open sides) as the oracle's [K][6] floats."""
    if cells is None:
        return None
    a = np.ascontiguousarray(np.asarray(cells, np.float32).reshape(K, 6))
    return a


def _sat(sat, H, W):
    a = np.ascontiguousarray(sat, np.uint8)
    if a.shape != (H, W):
        raise ValueError("sat must be [H, W] uint8")
    return a


def render_view(scene, offsets, cam, o: Opts | None = None, tile_mask=None, separable=False,
                order=None, cells=None, bounds=False, sat=None):
    """K contiguous subsets rendered and composited: dict(image, T, Cp, Tp, Dp, amb, sep,
    skip).  With `order` (front-to-back subset order) the partials are rendered in that
    order with saturation skipping (Sec. 4.2): a subset leaves empty the pixels whose prefix
    transmittance is below eps_comp, and skip[m, t] marks the tiles it left empty as a
    whole (no open pixel).  With
    `cells` (the subsets' k-d boxes [K, 2, 3]) cross-boundary Gaussians are filtered per
    ray as in Sec. 8.1.  With bounds: also "flip", the flip bounds of the ambiguous pixels:
    image and T of the composite, partC / partT / partD per partial (absolute amounts).
    With `sat` (with `order`; [H, W] uint8, the view's stale saturation state of Sec. 4.2
    step 2) the subset at rank r leaves pixel p empty exactly when r >= sat[p] (values >= K
    prune nothing), and the result adds "sat" (the state re-evaluated from this render for
    the next visit: the first rank after which the prefix transmittance is below eps_comp,
    255 for none) and "sat_amb" (pixels whose re-evaluation met a prefix within the
    AMB_SAT band); `separable` is not available then."""
    o = o or opts()
    k = _Keep(scene)
    c = camera(cam)
    off = np.ascontiguousarray(offsets, np.int64)
    K = off.size - 1
    H, W = cam.height, cam.width
    out = np.zeros((3, H, W)); To = np.ones((H, W))
    Cp = np.zeros((K, 3, H, W)); Tp = np.ones((K, H, W)); Dp = np.zeros((K, H, W))
    amb = np.zeros((H, W), np.uint8)
    sep = np.ones((H, W), np.uint8) if separable else None
    st = np.zeros(1, np.int64)
    tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
    od = _order(order, K)
    B = int(o.tile)
    skip = np.zeros((K, ((H + B - 1) // B) * ((W + B - 1) // B)), np.uint8)
    cl = _cells(cells, K)
    bd, bout = _bounds(H, W, K) if bounds else (None, None)
    if sat is not None:
        if od is None or separable:
            raise ValueError("sat needs order and excludes separable")
        si = _sat(sat, H, W)
        so = np.zeros((H, W), np.uint8)
        sa = np.zeros((H, W), np.uint8)
        rc = lib().orc_render_view_pruned(
            C.byref(k.p), _ptr(off), K, C.byref(c), C.byref(o), _ptr(tm), _ptr(od), _ptr(cl),
            _ptr(out), _ptr(To), _ptr(Cp), _ptr(Tp), _ptr(Dp), _ptr(amb), _ptr(skip), _ptr(st),
            C.byref(bd) if bd is not None else None, _ptr(si), _ptr(so), _ptr(sa))
        if rc != 0:
            raise ValueError("orc_render_view_pruned failed")
    else:
        lib().orc_render_view(C.byref(k.p), _ptr(off), K, C.byref(c), C.byref(o), _ptr(tm),
                              _ptr(od), _ptr(cl), _ptr(out), _ptr(To), _ptr(Cp), _ptr(Tp),
                              _ptr(Dp), _ptr(amb), _ptr(sep), _ptr(skip), _ptr(st),
                              C.byref(bd) if bd is not None else None)
    res = dict(image=out, T=To, Cp=Cp, Tp=Tp, Dp=Dp, amb=amb, sep=sep, skip=skip,
               evaluated=int(st[0]))
    if sat is not None:
        res["sat"], res["sat_amb"] = so, sa
    if bounds:
        res["flip"] = dict(image=bout["image"], T=bout["T"], partC=bout["partC"] * bd.cmax,
                           partT=bout["partT"], partD=bout["partC"] * bd.dmax, cmax=bd.cmax,
                           dmax=bd.dmax)
    return res


def backward_view(scene, offsets, cam, dLdC, dLdT=None, o: Opts | None = None, tile_mask=None,
                  order=None, cells=None, sat=None):
    """Gradients (float64) of sum(dLdC*C) + sum(dLdT*T) w.r.t. every parameter array
    (restricted to the pixels of tiles where tile_mask is nonzero, if given; with `order`,
    of the saturation-skipping render; with `order` and `sat`, of the render with that
    stale saturation state)."""
    o = o or opts()
    k = _Keep(scene)
    c = camera(cam)
    off = np.ascontiguousarray(offsets, np.int64)
    K = off.size - 1
    g = [np.zeros(a.shape) for a in scene.arrays()]
    gr = Grads(*(a.ctypes.data_as(_dp) for a in g))
    dC = np.ascontiguousarray(dLdC, np.float64)
    dT = None if dLdT is None else np.ascontiguousarray(dLdT, np.float64)
    tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
    cl = _cells(cells, K)
    if sat is not None:
        od = _order(order, K)
        if od is None:
            raise ValueError("sat needs order")
        rc = lib().orc_backward_view_pruned(C.byref(k.p), _ptr(off), K, C.byref(c), C.byref(o),
                                            _ptr(dC), _ptr(dT), _ptr(tm), _ptr(od), _ptr(cl),
                                            C.byref(gr), _ptr(_sat(sat, cam.height, cam.width)))
        if rc != 0:
            raise ValueError("orc_backward_view_pruned failed")
        return g
    lib().orc_backward_view(C.byref(k.p), _ptr(off), K, C.byref(c), C.byref(o), _ptr(dC), _ptr(dT),
                            _ptr(tm), _ptr(_order(order, K)), _ptr(cl), C.byref(gr))
    return g


def branch_stats(scene, offsets, cam, o: Opts | None = None):
    """Clamp branches of the adjoint that one view reaches: (flags[n], nclamp[n]).  flags:
    bit 0 / 1 the Jacobian's x / y clamp, bits 2-4 the colour clamp of r, g, b; nclamp: the
    pixels at which the Gaussian is blended with alpha held at alpha_max."""
    o = o or opts()
    k = _Keep(scene)
    c = camera(cam)
    off = np.ascontiguousarray(offsets, np.int64)
    flags = np.zeros(scene.n, np.int32)
    ncl = np.zeros(scene.n, np.int64)
    lib().orc_branch_stats(C.byref(k.p), _ptr(off), off.size - 1, C.byref(c), C.byref(o),
                           _ptr(flags), _ptr(ncl))
    return flags, ncl


def adam(p, g, m, v, lr, b1, b2, eps, step):
    """In-place FP64 Adam on float64 arrays."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(p.size, _ptr(p), _ptr(g), _ptr(m), _ptr(v), lr, b1, b2, eps, step)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def cell_order(boxes, eye):
    """Front-to-back order of k-d cells ([K, 2, 3] lo/hi boxes, infinite on unsplit sides)
    from `eye` (Sec. 4.2): an explicit stack of cell sets; each set is cut by the first
    axis-aligned plane (axes x, y, z, ascending coordinate) that leaves every cell of the
    set on one side, and the side holding the eye is taken first."""
    b = np.asarray(boxes, np.float64)
    eye = np.asarray(eye, np.float64)
    out = []
    stack = [list(range(b.shape[0]))]
    while stack:
        ids = stack.pop()
        if len(ids) == 1:
            out.append(ids[0])
            continue
        cut = None
        for ax in range(3):
            coords = np.unique(b[ids][:, :, ax])
            for p in coords[np.isfinite(coords)]:
                lo_side = [i for i in ids if b[i, 1, ax] <= p]
                hi_side = [i for i in ids if b[i, 0, ax] >= p]
                if lo_side and hi_side and len(lo_side) + len(hi_side) == len(ids):
                    cut = (lo_side, hi_side) if eye[ax] <= p else (hi_side, lo_side)
                    break
            if cut:
                break
        if cut is None:
            raise ValueError("not a k-d partition")
        stack.append(cut[1])  # popped after the whole first side
        stack.append(cut[0])
    return out


# ---------------------------------------------------------------- D-SSIM loss (Sec. 2, step 4)
# The photometric loss is L = (1 - lam) L1 + lam (1 - SSIM) (the paper's L_RGB + L_D-SSIM,
# read with the 3DGS convention lam = 0.2).  SSIM per channel with an 11 x 11 Gaussian
# window (sigma 1.5), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2; both terms
# are means over all pixels and channels of all views.
SSIM_C1, SSIM_C2 = 0.01 ** 2, 0.03 ** 2


def ssim_window(size=11, sigma=1.5):
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def _window_sum(a, w):
    """sum_{i,j} w[i] w[j] a[y + i - r, x + j - r] with zeros outside [H, W]."""
    r = len(w) // 2
    H, W = a.shape
    p = np.pad(a, r)
    h = sum(w[k] * p[:, k:k + W] for k in range(len(w)))
    return sum(w[k] * h[k:k + H, :] for k in range(len(w)))


def ssim_terms(x, y, w=None):
    """Per-pixel SSIM map S and its partial derivatives with respect to the local mean of x,
    the local mean of x^2 and the local mean of x y (one channel, FP64)."""
    w = ssim_window() if w is None else w
    mx, my = _window_sum(x, w), _window_sum(y, w)
    exx, eyy, exy = _window_sum(x * x, w), _window_sum(y * y, w), _window_sum(x * y, w)
    vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
    a1, a2 = 2 * mx * my + SSIM_C1, 2 * cxy + SSIM_C2
    b1, b2 = mx * mx + my * my + SSIM_C1, vx + vy + SSIM_C2
    S = a1 * a2 / (b1 * b2)
    dS_dmx = (2 * my * a2 - 2 * my * a1) / (b1 * b2) - S * 2 * mx / b1 + S * 2 * mx / b2
    dS_dexx = -S / b2
    dS_dexy = 2 * a1 / (b1 * b2)
    return S, dS_dmx, dS_dexx, dS_dexy


def loss_l1_dssim(imgs, tgts, lam=0.2):
    """(loss, [dL/dimg per view]) for lists of [3, H, W] images and targets (FP64)."""
    w = ssim_window()
    N = sum(a.size for a in imgs)
    l1 = sum(np.abs(np.asarray(a, np.float64) - b).sum() for a, b in zip(imgs, tgts)) / N
    ssum = 0.0
    grads = []
    for a, b in zip(imgs, tgts):
        a = np.asarray(a, np.float64)
        b = np.asarray(b, np.float64)
        g = (1.0 - lam) * np.sign(a - b) / N
        for ch in range(a.shape[0]):
            S, dmx, dexx, dexy = ssim_terms(a[ch], b[ch], w)
            ssum += S.sum()
            # the window is symmetric, so the adjoint of the windowed sum is itself
            dS = _window_sum(dmx, w) + 2 * a[ch] * _window_sum(dexx, w) + b[ch] * _window_sum(dexy, w)
            g[ch] -= lam * dS / N
        grads.append(g)
    loss = (1.0 - lam) * l1 + lam * (1.0 - ssum / N)
    return loss, grads
