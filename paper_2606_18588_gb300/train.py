"""Training step over the hot path: local render of K subsets for V views, global
composition, L1 loss, backward through both, Adam (Sec. 4.1 steps 1-3 and Sec. 2 step 4).

`BatchedStep` runs all V x K work of a step in one launch per stage (the batched path)
and can be captured as one CUDA graph; `PlainStep` launches per view and per subset (the
plain path).  `render` is the differentiable entry point for torch users.  Every stage
is a libsplx call; torch only owns the device buffers and the stream.
"""
from __future__ import annotations

import numpy as np
import torch

from . import splx as S

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")

# Per-group learning rates (means, log_scales, quats, opacity_logits, SH degree 0, SH higher);
# the paper names none, these are the customary 3DGS values.
DEFAULT_LR = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 2.5e-3 / 20.0)


def scene_to_device(scene) -> dict:
    return {k: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            for k, a in zip(GROUPS, scene.arrays())}


def city_to_device(layout, workers: int = 4, on_cell=None) -> dict:
    """Device parameter tensors of a CityLayout, generated one k-d cell at a time by
    `workers` spawned processes and copied into place, so the host holds a few cells at
    most.  on_cell(k, scene), if given, sees each cell's host arrays on the way."""
    import multiprocessing
    from .inputs import n_sh_coeffs
    N, nc = int(layout.offsets[-1]), n_sh_coeffs(layout.sh_degree)
    shapes = {"means": (N, 3), "log_scales": (N, 3), "quats": (N, 4), "opacity_logits": (N,),
              "sh": (N, nc, 3)}
    dev = {k: torch.empty(shapes[k], device="cuda") for k in GROUPS}
    with multiprocessing.get_context("spawn").Pool(workers) as pool:
        for k, sc in enumerate(pool.imap(layout.cell_scene, range(layout.K))):
            lo, hi = int(layout.offsets[k]), int(layout.offsets[k + 1])
            for name, arr in zip(GROUPS, sc.arrays()):
                dev[name][lo:hi].copy_(torch.from_numpy(arr))
            if on_cell is not None:
                on_cell(k, sc)
    torch.cuda.synchronize()
    return dev


def _subset_structs(dev, offsets, deg, mutable=False):
    f = S.params if mutable else S.gaussians
    return [f(*(dev[k][int(offsets[i]):int(offsets[i + 1])] for k in GROUPS), deg)
            for i in range(len(offsets) - 1)]


def _whole(dev, deg):
    return S.params(*(dev[k] for k in GROUPS), deg)


class BatchedStep:
    """One training step over a fixed batch of V views and K subsets."""

    def __init__(self, ctx: S.Context, params: dict, offsets, sh_degree: int, cams, targets,
                 opts: S.Opts | None = None, lr=DEFAULT_LR, pair_capacity: int = 0,
                 stream: torch.cuda.Stream | None = None, order=None, dssim: float = 0.0,
                 fused_adam: bool = True, stale: bool = False):
        """order: optional [V, K] front-to-back subset order per view, which turns on
        saturation skipping (visibility.orders_for_views gives it for k-d cells).
        stale: with an order, skip by each view's stale saturation state (Sec. 4.2 step 2)
        instead of the exact waves: one launch per stage, the state of this batch's views
        kept on the device and refreshed by every forward (reset by set_views).
        dssim: weight lambda of the D-SSIM term (0: plain L1).
        fused_adam: Adam runs inside the projection adjoint (no gradient arrays); False
        runs the backward into gradient arrays and a separate Adam pass (same result)."""
        self.dssim = float(dssim)
        self.fused_adam = bool(fused_adam)
        self.ctx, self.p, self.off, self.deg = ctx, params, np.asarray(offsets), sh_degree
        self.opts = opts or S.opts()
        self.stream = stream or torch.cuda.current_stream()
        self.g = None if self.fused_adam else {k: torch.zeros_like(v) for k, v in params.items()}
        self.m = {k: torch.zeros_like(v) for k, v in params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in params.items()}
        self.hp = S.adam_hp(lr, zero_grad=True)
        self.step_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.batch = S.Batch(ctx, _subset_structs(params, offsets, sh_degree), cams, self.opts,
                             pair_capacity, stream=self.stream)
        self.sat = None
        if order is not None:
            self.batch.set_order(order)
            if stale:
                self.sat = [torch.full((h * w,), 255, dtype=torch.uint8, device="cuda")
                            for h, w in self.batch.sizes]
                self.batch.set_stale(self.sat)
        self.rgb = torch.empty(self.batch.rgb_off[-1], device="cuda")
        self.dL = torch.empty_like(self.rgb)
        self.loss = torch.zeros(1, device="cuda")
        self.target = torch.empty_like(self.rgb)
        if targets is not None:
            self.set_targets(targets)
        if self.fused_adam:
            self._p_sub = _subset_structs(params, offsets, sh_degree, mutable=True)
            self._m_sub = _subset_structs(self.m, offsets, sh_degree, mutable=True)
            self._v_sub = _subset_structs(self.v, offsets, sh_degree, mutable=True)
        else:
            self._grads = _subset_structs(self.g, offsets, sh_degree, mutable=True)
        self.graph = None
        self.graphs = ()

    @property
    def pixels(self) -> int:
        return self.batch.total_pixels

    def set_targets(self, targets):
        """targets: list of [3,H,W] arrays/tensors, one per view, or one flat tensor."""
        if isinstance(targets, torch.Tensor) and targets.dim() == 1:
            self.target.copy_(targets, non_blocking=True)
            return
        flat = torch.cat([torch.as_tensor(t).reshape(-1) for t in targets])
        self.target.copy_(flat, non_blocking=True)

    def set_views(self, cams, order=None):
        """New camera poses (same resolutions, in the same order) and, with saturation
        skipping on, their front-to-back subset orders; a captured graph stays valid."""
        self.batch.set_cameras(cams, stream=self.stream)
        if order is not None:
            self.batch.set_order(order)
        if self.sat is not None:  # new poses: the states start over
            with torch.cuda.stream(self.stream):
                for t in self.sat:
                    t.fill_(255)
            self.batch.set_stale(self.sat)

    def run(self, events=None):
        """Forward, loss, backward, Adam on self.stream.  `events`, if given, is a list of
        5 CUDA events recorded around the stages (fwd | loss | bwd | adam)."""
        ev = events or [None] * 5
        self._forward(ev)
        self._update(ev)

    def _forward(self, ev):
        s = self.stream
        if ev[0] is not None: ev[0].record(s)
        self.batch.forward(self.rgb, None, stream=s)
        if ev[1] is not None: ev[1].record(s)

    def _update(self, ev):
        """Loss against self.target, backward, Adam."""
        s = self.stream
        if self.dssim > 0.0:
            self.batch.loss_l1_dssim(self.rgb, self.target, self.loss, self.dL, self.dssim, stream=s)
        else:
            S.loss_l1(self.ctx, self.rgb, self.target, self.loss, self.dL, stream=s)
        if ev[2] is not None: ev[2].record(s)
        if self.fused_adam:
            # backward and Adam in one pass (the adam interval ev[3] -> ev[4] is then empty)
            self.batch.backward_adam(self.dL, None, self._p_sub, self._m_sub, self._v_sub,
                                     self.hp, self.step_dev, stream=s)
            if ev[3] is not None: ev[3].record(s)
        else:
            self.batch.backward(self.dL, None, self._grads, stream=s)
            if ev[3] is not None: ev[3].record(s)
            S.step_device(self.ctx, _whole(self.p, self.deg), _whole(self.g, self.deg),
                          _whole(self.m, self.deg), _whole(self.v, self.deg), self.hp,
                          self.step_dev, stream=s)
        if ev[4] is not None: ev[4].record(s)

    def capture(self, events=None):
        """Captures run() as one CUDA graph on self.stream (the batch must already have
        run eagerly once, so its scratch exists; that run's counts decide whether the graph
        keeps the selected-prefix sort)."""
        self.batch.tune_prefix_sort(self.stream)
        S.graph_begin(self.ctx, self.stream)
        try:
            self.run(events)
        finally:
            g = S.graph_end(self.ctx, self.stream)
        self.graph = g
        return g

    def replay(self):
        self.graph.launch(self.stream)

    def capture_split(self):
        """Captures the step as two CUDA graphs, the forward and the rest (loss, backward,
        Adam), for step_from_host (the batch must already have run eagerly once)."""
        self.batch.tune_prefix_sort(self.stream)
        graphs = []
        for part in (self._forward, self._update):
            S.graph_begin(self.ctx, self.stream)
            try:
                part([None] * 5)
            finally:
                graphs.append(S.graph_end(self.ctx, self.stream))
        self.graphs = tuple(graphs)
        self._copy_stream = torch.cuda.Stream()
        self._copy_done = torch.cuda.Event()
        return self.graphs

    def step_from_host(self, host_target, host_loss=None):
        """One training step whose target images come from host memory (pinned, flat like
        self.target): the host-to-device copy runs on its own stream while the forward
        graph renders (the forward does not read the target), the rest of the step waits
        for it; the loss is copied back to host_loss (pinned, one float) if given.  Nothing
        waits on the host.  Needs capture_split()."""
        s, cs = self.stream, self._copy_stream
        cs.wait_stream(s)  # the previous step has finished reading self.target
        with torch.cuda.stream(cs):
            self.target.copy_(host_target, non_blocking=True)
            self._copy_done.record(cs)
        self.graphs[0].launch(s)
        s.wait_event(self._copy_done)
        self.graphs[1].launch(s)
        if host_loss is not None:
            with torch.cuda.stream(s):
                host_loss.copy_(self.loss, non_blocking=True)

    def status(self):
        return self.batch.status(self.stream)

    def close(self):
        if self.graph is not None:
            self.graph.close()
        for g in self.graphs:
            g.close()
        self.batch.close()


class PlainStep:
    """The same step launched per view: K render_partial calls, one composite, loss and
    backward per view, then one Adam update."""

    def __init__(self, ctx: S.Context, params: dict, offsets, sh_degree: int, cams, targets,
                 opts: S.Opts | None = None, lr=DEFAULT_LR, stream=None):
        self.ctx, self.p, self.off, self.deg, self.cams = ctx, params, np.asarray(offsets), sh_degree, cams
        self.opts = opts or S.opts()
        self.stream = stream or torch.cuda.current_stream()
        self.g = {k: torch.zeros_like(v) for k, v in params.items()}
        self.m = {k: torch.zeros_like(v) for k, v in params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in params.items()}
        self.hp = S.adam_hp(lr, zero_grad=True)
        self.step_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.targets = [torch.as_tensor(t).cuda().contiguous() for t in targets]
        self.subs = _subset_structs(params, offsets, sh_degree)
        self.grads = _subset_structs(self.g, offsets, sh_degree, mutable=True)
        self.parts = [[S.new_partial(c.height, c.width) for _ in self.subs] for c in cams]
        self.img = [torch.empty(3, c.height, c.width, device="cuda") for c in cams]
        self.dL = [torch.empty_like(i) for i in self.img]
        self.loss = torch.zeros(len(cams), device="cuda")

    @property
    def pixels(self) -> int:
        return sum(c.width * c.height for c in self.cams)

    def run(self):
        s = self.stream
        for v, cam in enumerate(self.cams):
            states = [S.render_partial(self.ctx, sub, cam, self.opts, self.parts[v][k], stream=s)
                      for k, sub in enumerate(self.subs)]
            S.composite(self.ctx, self.parts[v], cam.width, cam.height, self.opts, self.img[v],
                        None, stream=s)
            S.loss_l1(self.ctx, self.img[v], self.targets[v], self.loss[v:v + 1], self.dL[v],
                      stream=s)
            S.backward(self.ctx, self.subs, cam, self.parts[v], states, self.dL[v], None,
                       self.opts, self.grads, stream=s)
            for st in states:
                st.close(stream=s)
        S.step_device(self.ctx, _whole(self.p, self.deg), _whole(self.g, self.deg),
                      _whole(self.m, self.deg), _whole(self.v, self.deg), self.hp, self.step_dev,
                      stream=s)


# ---------------------------------------------------------------- autograd
class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, means, log_scales, quats, opacity_logits, sh):
        rgb, T = renderer._forward()
        ctx.renderer = renderer
        ctx.mark_non_differentiable(T)
        return rgb, T

    @staticmethod
    def backward(ctx, g_rgb, g_T):
        r = ctx.renderer
        grads = {k: torch.zeros_like(v) for k, v in r.p.items()}
        r._backward(g_rgb, g_T, grads)
        return (None, *(grads[k] for k in GROUPS))


class Renderer:
    """Differentiable batched render of V views x K subsets of fixed parameter tensors.

    render() returns the concatenated images (flat, layout from .views()) and total
    transmittance; backward of a loss on them fills .grad of the parameter tensors."""

    def __init__(self, ctx: S.Context, params: dict, offsets, sh_degree: int, cams,
                 opts: S.Opts | None = None, pair_capacity: int = 0):
        self.ctx, self.p, self.off, self.deg = ctx, params, np.asarray(offsets), sh_degree
        self.opts = opts or S.opts()
        self.batch = S.Batch(ctx, _subset_structs(params, offsets, sh_degree), cams, self.opts,
                             pair_capacity)

    def _forward(self):
        rgb = torch.empty(self.batch.rgb_off[-1], device="cuda")
        T = torch.empty(self.batch.total_pixels, device="cuda")
        self.batch.forward(rgb, T)
        return rgb, T

    def _backward(self, g_rgb, g_T, grads):
        g_rgb = torch.zeros(self.batch.rgb_off[-1], device="cuda") if g_rgb is None else g_rgb
        self.batch.backward(g_rgb.contiguous(), None if g_T is None else g_T.contiguous(),
                            _subset_structs(grads, self.off, self.deg, mutable=True))

    def render(self):
        return _RenderFn.apply(self, *(self.p[k] for k in GROUPS))

    def views(self, flat_rgb):
        return self.batch.views(flat_rgb)

    def close(self):
        self.batch.close()
