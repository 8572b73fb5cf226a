"""Python binding of libsplx (include/splx.h): argument marshalling only.

Every function here converts torch tensors / numpy cameras into the C structs of the ABI
and calls the library; all arithmetic of the path runs in the library's CUDA kernels.
There is no fallback: if libsplx.so is missing or fails to load, importing this module
raises.  Names follow the C entry points without the `splx_` prefix.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsplx.so")

OK, ERR_INVALID, ERR_BUDGET, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5, -6


class SplxError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.splx_strerror(code).decode()
        if code == ERR_CUDA:
            msg += f" ({_lib.splx_last_cuda_error().decode()})"
        super().__init__(f"{where}: {msg} [{code}]")


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsplx.so not built at {LIB_PATH}: run __graft_entry__.build() "
                      "(the CUDA path has no fallback)")
_lib = C.CDLL(LIB_PATH)


class Gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32)]


class Params(C.Structure):
    _fields_ = Gaussians._fields_


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_plane", C.c_float)]


class Opts(C.Structure):
    _fields_ = [("tile", C.c_int32), ("eps_T", C.c_float), ("eps_comp", C.c_float),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("bg", C.c_float * 3)]


class Partial(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("T", C.c_void_p), ("depth", C.c_void_p), ("last", C.c_void_p)]


class Adam(C.Structure):
    _fields_ = [("lr", C.c_float * 6), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("zero_grad", C.c_int32)]


_P = C.c_void_p
_sigs = {
    "splx_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_size_t]),
    "splx_destroy": (C.c_int, [_P]),
    "splx_scratch_bytes": (C.c_size_t, [_P]),
    "splx_render_partial": (C.c_int, [_P, _P, _P, _P, _P, C.POINTER(_P), _P]),
    "splx_composite": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, _P]),
    "splx_backward": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P]),
    "splx_state_release": (C.c_int, [_P, _P, _P]),
    "splx_state_export": (C.c_int, [_P, _P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _P, _P, _P,
                                    _P]),
    "splx_step": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int64, _P]),
    "splx_step_device": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "splx_loss_l1": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P]),
    "splx_batch_create": (C.c_int, [_P, _P, C.c_int32, _P, C.c_int32, _P, C.c_int64,
                                    C.POINTER(_P), _P]),
    "splx_batch_set_cameras": (C.c_int, [_P, _P, C.c_int32, _P]),
    "splx_batch_layout": (C.c_int, [_P, _P, _P]),
    "splx_batch_forward": (C.c_int, [_P, _P, _P, _P]),
    "splx_batch_backward": (C.c_int, [_P, _P, _P, _P, _P]),
    "splx_batch_backward_adam": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "splx_batch_status": (C.c_int, [_P, C.POINTER(C.c_int64), _P]),
    "splx_batch_destroy": (C.c_int, [_P]),
    "splx_batch_set_timing": (C.c_int, [_P, C.c_int]),
    "splx_batch_kernel_times": (C.c_int, [_P, _P]),
    "splx_batch_counters": (C.c_int, [_P, _P, _P]),
    "splx_batch_set_launch": (C.c_int, [_P, C.c_int32]),
    "splx_batch_set_order": (C.c_int, [_P, _P]),
    "splx_batch_set_stale": (C.c_int, [_P, _P]),
    "splx_batch_visible": (C.c_int, [_P, C.POINTER(C.c_int64), _P]),
    "splx_batch_set_visibility": (C.c_int, [_P, C.c_int32]),
    "splx_batch_set_prefix_sort": (C.c_int, [_P, C.c_int32]),
    "splx_batch_tune_prefix_sort": (C.c_int, [_P, _P]),
    "splx_batch_set_cross_filter": (C.c_int, [_P, _P]),
    "splx_batch_loss_l1_dssim": (C.c_int, [_P, _P, _P, C.c_float, _P, _P, _P]),
    "splx_loss_l1_dssim": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, C.c_float, _P, _P, _P]),
    "splx_batch_max_ctas_per_sm": (C.c_int, [_P, _P, _P]),
    "splx_server_create": (C.c_int, [_P, _P, C.c_int32, _P, C.c_size_t, C.c_int32, C.c_int32,
                                     C.POINTER(_P)]),
    "splx_server_submit": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_int64)]),
    "splx_server_poll": (C.c_int, [_P, _P, _P, C.c_int32, C.POINTER(C.c_int32)]),
    "splx_server_stats": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_size_t)]),
    "splx_server_destroy": (C.c_int, [_P]),
    "splx_graph_begin": (C.c_int, [_P, _P]),
    "splx_graph_end": (C.c_int, [_P, _P, C.POINTER(_P)]),
    "splx_graph_launch": (C.c_int, [_P, _P]),
    "splx_view_regions": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P]),
    "splx_render_partial_filtered": (C.c_int, [_P, _P, C.c_int32, C.c_int32, _P, _P, _P, _P,
                                               _P, _P, _P]),
    "splx_server_request_times": (C.c_int, [_P, C.c_int64, _P]),
    "splx_graph_set_timing_ring": (C.c_int, [_P, C.c_int32]),
    "splx_batch_kernel_times_slot": (C.c_int, [_P, _P, C.c_int32, _P]),
    "splx_graph_destroy": (C.c_int, [_P]),
    "splx_render_partial_noalloc": (C.c_int, [_P, _P, _P, _P, _P]),
    "splx_device_status": (C.c_int, [_P, _P]),
    "splx_strerror": (C.c_char_p, [C.c_int]),
    "splx_last_cuda_error": (C.c_char_p, []),
    "splx_launch_count": (C.c_int64, [_P]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sigs)


def _check(code, where):
    if code != OK:
        raise SplxError(code, where)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or t.dtype not in (torch.float32, torch.int32) or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA float32/int32 tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- struct helpers
def gaussians(means, log_scales, quats, opacity_logits, sh, sh_degree) -> Gaussians:
    n = means.shape[0]
    return Gaussians(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh),
                     n, sh_degree)


def params(means, log_scales, quats, opacity_logits, sh, sh_degree) -> Params:
    return Params(*[getattr(gaussians(means, log_scales, quats, opacity_logits, sh, sh_degree), f)
                    for f, _ in Gaussians._fields_])


def camera(cam) -> Camera:
    c = Camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).reshape(-1)]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32).reshape(-1)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height, c.near_plane = cam.width, cam.height, cam.near
    return c


def opts(tile=16, eps_T=1e-4, eps_comp=1e-4, alpha_min=1.0 / 255.0, alpha_max=0.99,
         bg=(0.0, 0.0, 0.0)) -> Opts:
    o = Opts()
    o.tile, o.eps_T, o.eps_comp, o.alpha_min, o.alpha_max = tile, eps_T, eps_comp, alpha_min, alpha_max
    o.bg[:] = list(bg)
    return o


# ---------------------------------------------------------------- context
class Context:
    """A libsplx context on one CUDA device (scratch pool + HBM budget)."""

    def __init__(self, device: int | None = None, hbm_budget_bytes: int = 0):
        self.device = torch.cuda.current_device() if device is None else device
        h = C.c_void_p()
        _check(_lib.splx_create(C.byref(h), self.device, hbm_budget_bytes), "splx_create")
        self.h = h
        self._lock = threading.Lock()

    def close(self):
        if self.h:
            _lib.splx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def scratch_bytes(self) -> int:
        return int(_lib.splx_scratch_bytes(self.h))

    @property
    def launch_count(self) -> int:
        return int(_lib.splx_launch_count(self.h))

    def device_status(self, stream=None) -> int:
        return int(_lib.splx_device_status(self.h, _stream(stream)))


class State:
    """Forward state of one (view, subset) render, released on close/garbage collection."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def export(self, stream=None):
        """(ranges [n_tiles,2] uint32, sorted keys [n_pairs] uint64 (depth bits << 32 |
        index), records [n,16] f32) as CPU numpy arrays."""
        npairs, ntiles = C.c_int64(), C.c_int64()
        _check(_lib.splx_state_export(self.ctx.h, self.h, C.byref(npairs), C.byref(ntiles), None,
                                      None, None, _stream(stream)), "splx_state_export")
        n = _lib_state_n(self)
        ranges = torch.empty(max(ntiles.value, 1) * 2, dtype=torch.int32, device="cuda")
        keys = torch.empty(max(npairs.value, 1) * 2, dtype=torch.int32, device="cuda")
        rec = torch.empty(max(n, 1) * 16, dtype=torch.float32, device="cuda")
        _check(_lib.splx_state_export(self.ctx.h, self.h, None, None, _ptr(ranges), _ptr(keys),
                                      _ptr(rec), _stream(stream)), "splx_state_export")
        r = ranges.cpu().numpy().view(np.uint32)[:2 * ntiles.value].reshape(-1, 2)
        v = keys.cpu().numpy().view(np.uint64)[:npairs.value]
        return r, v, rec.cpu().numpy()[:16 * n].reshape(-1, 16)

    def close(self, stream=None):
        if self.h:
            _lib.splx_state_release(self.ctx.h, self.h, _stream(stream))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _lib_state_n(state) -> int:
    return state.n


def new_partial(H, W, device=None):
    dev = device or torch.device("cuda")
    return dict(rgb=torch.empty(3, H, W, device=dev), T=torch.empty(H, W, device=dev),
                depth=torch.empty(H, W, device=dev),
                last=torch.empty(H, W, device=dev, dtype=torch.int32))


def _partial_struct(p) -> Partial:
    return Partial(_ptr(p["rgb"]), _ptr(p["T"]), _ptr(p["depth"]), _ptr(p["last"]))


# ---------------------------------------------------------------- per-view entry points
def view_regions(ctx: Context, subsets, cam, o: Opts, stream=None) -> np.ndarray:
    """Every subset's visible region and depth range in one view ([K, 6] uint32), the input
    of the per-view cross-boundary filter."""
    c = cam if isinstance(cam, Camera) else camera(cam)
    K = len(subsets)
    sarr = (Gaussians * K)(*subsets)
    out = np.zeros((K, 6), np.uint32)
    _check(_lib.splx_view_regions(ctx.h, sarr, K, C.byref(c), C.byref(o),
                                  out.ctypes.data_as(C.c_void_p), _stream(stream)),
           "splx_view_regions")
    return out


def render_partial(ctx: Context, subset: Gaussians, cam, o: Opts, out: dict, keep_state=True,
                   stream=None, cross=None):
    """Local render of one subset into `out` (a new_partial dict); returns a State.
    cross = (k, cells [K, 2, 3], regions [K, 6]) turns on cross-boundary filtering with this
    subset as cell k (regions from view_regions for the same camera)."""
    c = cam if isinstance(cam, Camera) else camera(cam)
    h = C.c_void_p()
    ps = _partial_struct(out)
    if cross is None:
        _check(_lib.splx_render_partial(ctx.h, C.byref(subset), C.byref(c), C.byref(o),
                                        C.byref(ps), C.byref(h) if keep_state else None,
                                        _stream(stream)), "splx_render_partial")
    else:
        k, cells, regions = cross
        cl = np.ascontiguousarray(np.asarray(cells, np.float32).reshape(-1, 6))
        rg = np.ascontiguousarray(np.asarray(regions, np.uint32).reshape(-1, 6))
        if cl.shape[0] != rg.shape[0]:
            raise ValueError("cells and regions must describe the same K subsets")
        _check(_lib.splx_render_partial_filtered(
            ctx.h, C.byref(subset), int(k), cl.shape[0], cl.ctypes.data_as(C.c_void_p),
            rg.ctypes.data_as(C.c_void_p), C.byref(c), C.byref(o), C.byref(ps),
            C.byref(h) if keep_state else None, _stream(stream)), "splx_render_partial_filtered")
    if not keep_state:
        return None
    st = State(ctx, h)
    st.n = int(subset.n)
    return st


def render_partial_noalloc(subset: Gaussians, cam, o: Opts, out: dict, stream=None):
    """Local render of one subset without any device allocation, for callers that cannot
    allocate (their HBM is held by another allocator, or cudaMalloc's implicit
    synchronisation is not allowed in their loop).  Uses the library's fixed 32 MiB
    scratch array; limits and sharing rules are those of splx_render_partial_noalloc."""
    c = cam if isinstance(cam, Camera) else camera(cam)
    ps = _partial_struct(out)
    _check(_lib.splx_render_partial_noalloc(C.byref(subset), C.byref(c), C.byref(o), C.byref(ps),
                                            _stream(stream)), "splx_render_partial_noalloc")


def composite(ctx: Context, parts, W, H, o: Opts, out_rgb, out_T=None, stream=None):
    arr = (Partial * len(parts))(*[_partial_struct(p) for p in parts])
    _check(_lib.splx_composite(ctx.h, arr, len(parts), W, H, C.byref(o), _ptr(out_rgb),
                               _ptr(out_T), _stream(stream)), "splx_composite")


def backward(ctx: Context, subsets, cam, parts, states, dL_drgb, dL_dT, o: Opts, grads,
             stream=None):
    K = len(subsets)
    c = cam if isinstance(cam, Camera) else camera(cam)
    sarr = (Gaussians * K)(*subsets)
    parr = (Partial * K)(*[_partial_struct(p) for p in parts])
    starr = (C.c_void_p * K)(*[s.h for s in states])
    garr = (Params * K)(*grads)
    _check(_lib.splx_backward(ctx.h, sarr, K, C.byref(c), parr, starr, _ptr(dL_drgb), _ptr(dL_dT),
                              C.byref(o), garr, _stream(stream)), "splx_backward")


def adam_hp(lr, betas=(0.9, 0.999), eps=1e-15, zero_grad=False) -> Adam:
    hp = Adam()
    hp.lr[:] = list(lr)
    hp.beta1, hp.beta2, hp.eps, hp.zero_grad = betas[0], betas[1], eps, int(bool(zero_grad))
    return hp


def step(ctx: Context, p: Params, g: Params, m: Params, v: Params, lr, step_idx, betas=(0.9, 0.999),
         eps=1e-15, zero_grad=False, stream=None):
    hp = adam_hp(lr, betas, eps, zero_grad)
    _check(_lib.splx_step(ctx.h, C.byref(p), C.byref(g), C.byref(m), C.byref(v), C.byref(hp),
                          int(step_idx), _stream(stream)), "splx_step")


def step_device(ctx: Context, p: Params, g: Params, m: Params, v: Params, hp: Adam, step_dev,
                stream=None):
    """Adam with the step counter in device memory (an int64 CUDA tensor of one element)."""
    if step_dev.dtype != torch.int64 or not step_dev.is_cuda:
        raise ValueError("step_dev must be a CUDA int64 tensor")
    _check(_lib.splx_step_device(ctx.h, C.byref(p), C.byref(g), C.byref(m), C.byref(v),
                                 C.byref(hp), C.c_void_p(step_dev.data_ptr()), _stream(stream)),
           "splx_step_device")


def loss_l1(ctx: Context, img, target, loss_out, dL_dimg=None, stream=None):
    _check(_lib.splx_loss_l1(ctx.h, _ptr(img), _ptr(target), img.numel(), _ptr(loss_out),
                             _ptr(dL_dimg), _stream(stream)), "splx_loss_l1")


def loss_l1_dssim(ctx: Context, img, target, loss_out, dL_dimg, lam=0.2, stream=None):
    """(1 - lam) L1 + lam (1 - SSIM) of one [3, H, W] image."""
    _, H, W = img.shape
    _check(_lib.splx_loss_l1_dssim(ctx.h, _ptr(img), _ptr(target), int(W), int(H), float(lam),
                                   _ptr(loss_out), _ptr(dL_dimg), _stream(stream)),
           "splx_loss_l1_dssim")


# ---------------------------------------------------------------- batched path
class Server:
    """Render server over K resident subsets: continuous batching of camera requests
    of any resolution, admission by an HBM budget, launches overlapping on `slots`
    streams.  submit() takes the device output tensor [3,H,W]; poll() returns the
    (id, status) pairs finished since the last call."""

    def __init__(self, ctx: Context, subsets, o: Opts, hbm_budget_bytes: int, slots: int = 4,
                 max_views: int = 8):
        self.ctx = ctx
        self.K = len(subsets)
        self._subsets = (Gaussians * self.K)(*subsets)
        h = C.c_void_p()
        _check(_lib.splx_server_create(ctx.h, self._subsets, self.K, C.byref(o),
                                       int(hbm_budget_bytes), int(slots), int(max_views),
                                       C.byref(h)), "splx_server_create")
        self.h = h
        self._outs = {}  # id -> output tensor, kept alive until the request finishes
        self._ids = (C.c_int64 * 256)()
        self._st = (C.c_int32 * 256)()

    def submit(self, cam, out_rgb, order=None) -> int:
        """order: optional front-to-back subset order for this camera (saturation skipping)."""
        c = cam if isinstance(cam, Camera) else camera(cam)
        if tuple(out_rgb.shape) != (3, c.height, c.width):
            raise ValueError("out_rgb must be [3, H, W]")
        rid = C.c_int64()
        op = None
        if order is not None:
            oa = np.ascontiguousarray(order, np.int32)
            if oa.shape != (self.K,):
                raise ValueError(f"order must have {self.K} entries")
            op = oa.ctypes.data_as(C.c_void_p)
        _check(_lib.splx_server_submit(self.h, C.byref(c), op, _ptr(out_rgb), C.byref(rid)),
               "splx_server_submit")
        self._outs[rid.value] = out_rgb
        return rid.value

    def poll(self):
        done = []
        while True:
            n = C.c_int32()
            _check(_lib.splx_server_poll(self.h, self._ids, self._st, 256, C.byref(n)),
                   "splx_server_poll")
            for i in range(n.value):
                self._outs.pop(self._ids[i], None)
                done.append((self._ids[i], self._st[i]))
            if n.value < 256:
                return done

    def request_times(self, rid: int) -> dict:
        """Device timeline of a finished request, ms after the server's creation."""
        arr = (C.c_float * 3)()
        _check(_lib.splx_server_request_times(self.h, int(rid), arr), "splx_server_request_times")
        return {"begin": arr[0], "counted": arr[1], "end": arr[2]}

    def stats(self):
        q, f, r = C.c_int32(), C.c_int32(), C.c_size_t()
        _check(_lib.splx_server_stats(self.h, C.byref(q), C.byref(f), C.byref(r)),
               "splx_server_stats")
        return {"queued": q.value, "inflight": f.value, "reserved_bytes": r.value}

    def close(self):
        if self.h:
            _lib.splx_server_destroy(self.h)
            self.h = None
            self._outs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A planned batch of V views x K subsets (persistent scratch, capturable runs)."""

    def __init__(self, ctx: Context, subsets, cams, o: Opts, pair_capacity=0, stream=None):
        self.ctx = ctx
        self.K, self.V = len(subsets), len(cams)
        self._subsets = (Gaussians * self.K)(*subsets)
        self._cams = (Camera * self.V)(*[c if isinstance(c, Camera) else camera(c) for c in cams])
        self.sizes = [(c.height, c.width) for c in self._cams]
        h = C.c_void_p()
        _check(_lib.splx_batch_create(ctx.h, self._subsets, self.K, self._cams, self.V, C.byref(o),
                                      int(pair_capacity), C.byref(h), _stream(stream)),
               "splx_batch_create")
        self.h = h
        rgb_off = (C.c_int64 * (self.V + 1))()
        pix_off = (C.c_int64 * (self.V + 1))()
        _check(_lib.splx_batch_layout(self.h, rgb_off, pix_off), "splx_batch_layout")
        self.rgb_off = list(rgb_off)
        self.pix_off = list(pix_off)

    @property
    def total_pixels(self) -> int:
        return self.pix_off[-1]

    def set_cameras(self, cams, stream=None):
        arr = (Camera * self.V)(*[c if isinstance(c, Camera) else camera(c) for c in cams])
        _check(_lib.splx_batch_set_cameras(self.h, arr, self.V, _stream(stream)),
               "splx_batch_set_cameras")

    def forward(self, out_rgb, out_T=None, stream=None):
        _check(_lib.splx_batch_forward(self.h, _ptr(out_rgb), _ptr(out_T), _stream(stream)),
               "splx_batch_forward")

    def backward(self, dL_drgb, dL_dT, grads, stream=None):
        garr = (Params * self.K)(*grads)
        _check(_lib.splx_batch_backward(self.h, _ptr(dL_drgb), _ptr(dL_dT), garr, _stream(stream)),
               "splx_batch_backward")

    def backward_adam(self, dL_drgb, dL_dT, params, m, v, hp: Adam, step_dev, stream=None):
        """Backward with Adam fused into the projection adjoint: params[k] (the subsets the
        batch was created on), m[k] and v[k] are updated in place; step_dev is a CUDA int64
        tensor of one element, incremented first."""
        if step_dev.dtype != torch.int64 or not step_dev.is_cuda:
            raise ValueError("step_dev must be a CUDA int64 tensor")
        parr = (Params * self.K)(*params)
        marr = (Params * self.K)(*m)
        varr = (Params * self.K)(*v)
        _check(_lib.splx_batch_backward_adam(self.h, _ptr(dL_drgb), _ptr(dL_dT), parr, marr, varr,
                                             C.byref(hp), C.c_void_p(step_dev.data_ptr()),
                                             _stream(stream)),
               "splx_batch_backward_adam")

    def status(self, stream=None):
        pairs = C.c_int64()
        code = _lib.splx_batch_status(self.h, C.byref(pairs), _stream(stream))
        return code, int(pairs.value)

    KERNELS = ("project", "scan", "fill", "sort", "raster_fwd", "composite", "composite_bwd",
               "raster_bwd", "project_bwd")

    def set_timing(self, enable=True):
        _check(_lib.splx_batch_set_timing(self.h, int(bool(enable))), "splx_batch_set_timing")

    def kernel_times(self, graph=None, slot=None) -> dict:
        """Per-kernel ms of the last run, or of the replay of `graph` that took ring `slot`."""
        arr = (C.c_float * len(self.KERNELS))()
        if graph is None:
            _check(_lib.splx_batch_kernel_times(self.h, arr), "splx_batch_kernel_times")
        else:
            _check(_lib.splx_batch_kernel_times_slot(self.h, graph.h, int(slot), arr),
                   "splx_batch_kernel_times_slot")
        return dict(zip(self.KERNELS, [float(x) for x in arr]))

    def set_launch(self, raster_ctas_per_sm: int):
        """0: one rasteriser CTA per work item; n > 0: n persistent CTAs per SM."""
        _check(_lib.splx_batch_set_launch(self.h, int(raster_ctas_per_sm)), "splx_batch_set_launch")

    def loss_l1_dssim(self, rgb, target, loss, dL, lam=0.2, stream=None):
        """(1 - lam) L1 + lam (1 - SSIM) over the batch's views into loss[0], gradient into dL."""
        _check(_lib.splx_batch_loss_l1_dssim(self.h, _ptr(rgb), _ptr(target), float(lam), _ptr(loss),
                                             _ptr(dL), _stream(stream)), "splx_batch_loss_l1_dssim")

    def set_visibility(self, enable: bool):
        """Spatial visibility regions on (default) or off; results are identical."""
        _check(_lib.splx_batch_set_visibility(self.h, int(bool(enable))),
               "splx_batch_set_visibility")

    def set_prefix_sort(self, enable: bool):
        """Selected-prefix sort of long tile segments on (default) or off; results are
        identical."""
        _check(_lib.splx_batch_set_prefix_sort(self.h, int(bool(enable))),
               "splx_batch_set_prefix_sort")

    def tune_prefix_sort(self, stream=None):
        """Keeps the selected-prefix sort only if the last eager forward handed at most a
        quarter of its prefix items back to the whole sort (synchronises)."""
        _check(_lib.splx_batch_tune_prefix_sort(self.h, _stream(stream)),
               "splx_batch_tune_prefix_sort")

    def set_cross_filter(self, cells):
        """Cross-boundary per-ray filtering with the subsets' k-d boxes [K, 2, 3] (lo, hi;
        infinite on open sides), or off (None); see splx_batch_set_cross_filter."""
        if cells is None:
            _check(_lib.splx_batch_set_cross_filter(self.h, None), "splx_batch_set_cross_filter")
            return
        a = np.ascontiguousarray(np.asarray(cells, np.float32).reshape(self.K, 6))
        _check(_lib.splx_batch_set_cross_filter(self.h, a.ctypes.data_as(C.c_void_p)),
               "splx_batch_set_cross_filter")

    def set_order(self, order):
        """Saturation skipping with a [V, K] front-to-back subset order per view (None:
        off); see splx_batch_set_order."""
        if order is None:
            _check(_lib.splx_batch_set_order(self.h, None), "splx_batch_set_order")
            return
        a = np.ascontiguousarray(order, np.int32)
        if a.shape != (self.V, self.K):
            raise ValueError(f"order must be [{self.V}, {self.K}]")
        _check(_lib.splx_batch_set_order(self.h, a.ctypes.data_as(C.c_void_p)),
               "splx_batch_set_order")

    def set_stale(self, planes):
        """Stale saturation state: `planes` is a list of V uint8 CUDA tensors, plane v of
        H_v * W_v elements (255: nothing pruned), kept alive by the caller and rewritten by
        every forward; None turns it off.  See splx_batch_set_stale."""
        if planes is None:
            _check(_lib.splx_batch_set_stale(self.h, None), "splx_batch_set_stale")
            self._stale = None
            return
        if len(planes) != self.V:
            raise ValueError(f"need {self.V} planes")
        for t, (h, w) in zip(planes, self.sizes):
            if t.dtype != torch.uint8 or not t.is_cuda or t.numel() != h * w or not t.is_contiguous():
                raise ValueError("each plane must be a contiguous CUDA uint8 tensor of H*W")
        arr = (C.c_void_p * self.V)(*[t.data_ptr() for t in planes])
        _check(_lib.splx_batch_set_stale(self.h, arr), "splx_batch_set_stale")
        self._stale = list(planes)

    def max_ctas_per_sm(self) -> tuple[int, int]:
        f, b = C.c_int32(0), C.c_int32(0)
        _check(_lib.splx_batch_max_ctas_per_sm(self.h, C.byref(f), C.byref(b)),
               "splx_batch_max_ctas_per_sm")
        return f.value, b.value

    def counters(self, stream=None) -> dict:
        arr = (C.c_int64 * 11)()
        _check(_lib.splx_batch_counters(self.h, arr, _stream(stream)), "splx_batch_counters")
        return dict(pairs=arr[0], entries_fwd=arr[1], alpha_fwd=arr[2], blended=arr[3],
                    entries_bwd=arr[4], alpha_bwd=arr[5], contrib_bwd=arr[6],
                    skipped_items=arr[7], outside_items=arr[8], prefix_items=arr[9],
                    retried_items=arr[10])

    def visible(self, stream=None) -> int:
        """(view, Gaussian) pairs the last forward's projection kept (synchronises)."""
        n = C.c_int64()
        _check(_lib.splx_batch_visible(self.h, C.byref(n), _stream(stream)), "splx_batch_visible")
        return int(n.value)

    def views(self, flat_rgb):
        """Split a concatenated rgb buffer into per-view [3,H,W] tensors."""
        return [flat_rgb[self.rgb_off[v]:self.rgb_off[v + 1]].view(3, *self.sizes[v])
                for v in range(self.V)]

    def close(self):
        if self.h:
            _lib.splx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A CUDA graph of library calls captured on one stream."""

    def __init__(self, h):
        self.h = h

    def launch(self, stream=None):
        _check(_lib.splx_graph_launch(self.h, _stream(stream)), "splx_graph_launch")

    def set_timing_ring(self, slots: int):
        """Launch i records the graph's timing events into ring slot i mod slots."""
        _check(_lib.splx_graph_set_timing_ring(self.h, int(slots)), "splx_graph_set_timing_ring")

    def close(self):
        if self.h:
            _lib.splx_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def graph_begin(ctx: Context, stream):
    _check(_lib.splx_graph_begin(ctx.h, _stream(stream)), "splx_graph_begin")


def graph_end(ctx: Context, stream) -> Graph:
    h = C.c_void_p()
    _check(_lib.splx_graph_end(ctx.h, _stream(stream), C.byref(h)), "splx_graph_end")
    return Graph(h)
