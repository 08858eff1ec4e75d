"""Rendering front end: workspace management and the autograd Function.

PyTorch supplies device memory (every buffer is a torch tensor handed to the
C ABI as a pointer) and the current CUDA stream; the library does the rest.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import sgsplat as _sg
from .sgsplat import DeviceScene, SGError

# Last pair count seen per (scene size, camera sizes): sizes the next
# workspace so that a steady stream of renders needs no second attempt.
_PAIR_HINT: dict = {}
PAIR_HEADROOM = 1.05


def _key(scene, cams):
    return (scene.n, scene.n_lobes, tuple((int(c.width), int(c.height)) for c in cams))


@dataclass
class ForwardOut:
    img: torch.Tensor        # [V,3,H,W] (equal view sizes) or flat [3*sum HW]
    T_final: torch.Tensor    # [V,H,W] or flat
    last: torch.Tensor       # [V,H,W] or flat, int32
    ws: torch.Tensor         # uint8 workspace the backward reads
    sizes: dict


def _alloc_outputs(cams, device):
    same = all((c.width, c.height) == (cams[0].width, cams[0].height) for c in cams)
    if same:
        V, H, W = len(cams), int(cams[0].height), int(cams[0].width)
        return (torch.empty(V, 3, H, W, device=device), torch.empty(V, H, W, device=device),
                torch.empty(V, H, W, dtype=torch.int32, device=device))
    P = sum(int(c.width) * int(c.height) for c in cams)
    return (torch.empty(3 * P, device=device), torch.empty(P, device=device),
            torch.empty(P, dtype=torch.int32, device=device))


def render_forward(scene: DeviceScene, cams, stream=None, importance=None) -> ForwardOut:
    """Plain forward. importance: optional float32 [N] tensor that receives the
    per-Gaussian importance score (sum of alpha T over the views' pixels)."""
    device = scene.means.device
    img, T, last = _alloc_outputs(cams, device)
    key = _key(scene, cams)
    hint = _PAIR_HINT.get(key)
    if hint is None:
        hint = 8 * scene.n * len(cams)

    def call(ws):
        if importance is None:
            return _sg.sg_render_forward(scene, cams, ws, img, T, last, stream, raise_on_error=False)
        return _sg.sg_render_forward_importance(scene, cams, ws, img, T, last, importance, stream,
                                                raise_on_error=False)

    sizes = _sg.sg_workspace_query(scene, cams, int(hint * PAIR_HEADROOM) + 1024)
    ws = torch.empty(sizes["ws_bytes"], dtype=torch.uint8, device=device)
    st, out = call(ws)
    if st == _sg.SG_ERR_CAPACITY:
        sizes = _sg.sg_workspace_query(scene, cams, int(out["n_pairs"] * PAIR_HEADROOM) + 1024)
        ws = torch.empty(sizes["ws_bytes"], dtype=torch.uint8, device=device)
        st, out = call(ws)
    if st != _sg.SG_OK:
        raise SGError(st, _sg.sg_last_error())
    _PAIR_HINT[key] = out["n_pairs"]
    return ForwardOut(img, T, last, ws, out)


def alloc_grads(scene: DeviceScene):
    return {k: torch.empty(getattr(scene, k).shape, dtype=torch.float32, device=scene.means.device)
            for k in scene.grad_fields()}


def render_backward(scene: DeviceScene, cams, fwd: ForwardOut, d_img, grads=None, stream=None):
    """Gradients of sum(d_img * img) for every float input (binary32 tensors)."""
    if grads is None:
        grads = alloc_grads(scene)
    bwd = torch.empty(fwd.sizes["bwd_ws_bytes"], dtype=torch.uint8, device=scene.means.device)
    _sg.sg_render_backward(scene, cams, fwd.ws, fwd.T_final, fwd.last, d_img.contiguous(), bwd,
                           grads, stream)
    return grads


class HostStep:
    """One forward + backward of a scene whose parameters and upstream gradient
    live in pinned host memory, with the image and every gradient copied back
    (a host-side training or serving loop).

    Copies that do not gate the next kernel overlap with it on a second stream:
    the upstream gradient goes up while the forward runs and the image comes
    down while the backward runs. The scene's parameters go up before the
    forward and the gradients come down after the backward, on the caller's
    stream; __call__ returns once everything is back on the host.
    """

    def __init__(self, scene: DeviceScene, cams, host_scene: dict, host_d_img, host_img, host_grads: dict):
        self.scene, self.cams = scene, cams
        self.host_scene, self.host_d_img = host_scene, host_d_img
        self.host_img, self.host_grads = host_img, host_grads
        dev = scene.means.device
        self.d_img = torch.empty(host_d_img.shape, dtype=host_d_img.dtype, device=dev)
        self.grads = alloc_grads(scene)
        self.side = torch.cuda.Stream(device=dev)

    def bytes_moved(self):
        up = sum(t.numel() * t.element_size() for t in self.host_scene.values())
        up += self.host_d_img.numel() * self.host_d_img.element_size()
        down = self.host_img.numel() * self.host_img.element_size()
        down += sum(t.numel() * t.element_size() for t in self.host_grads.values())
        return up, down

    def __call__(self):
        main = torch.cuda.current_stream()
        for k, t in self.host_scene.items():
            getattr(self.scene, k).copy_(t, non_blocking=True)
        self.side.wait_stream(main)
        with torch.cuda.stream(self.side):
            self.d_img.copy_(self.host_d_img, non_blocking=True)
            d_img_ready = self.side.record_event()
        out = render_forward(self.scene, self.cams)
        self.side.wait_stream(main)
        with torch.cuda.stream(self.side):
            self.host_img.copy_(out.img.view(self.host_img.shape), non_blocking=True)
        out.img.record_stream(self.side)
        main.wait_event(d_img_ready)
        render_backward(self.scene, self.cams, out, self.d_img, self.grads)
        for k, t in self.host_grads.items():
            t.copy_(self.grads[k], non_blocking=True)
        main.synchronize()
        self.side.synchronize()
        return self.host_img, self.host_grads


@dataclass
class _Slot:
    scene: DeviceScene
    grads: dict
    d_img: torch.Tensor | None = None
    bwd_done: torch.cuda.Event | None = None    # last step using the slot finished its backward
    down_done: torch.cuda.Event | None = None   # ... and its gradients are on the host


class PipelinedStep:
    """Handle of one queued HostPipeline step."""

    def __init__(self, done: torch.cuda.Event, host_img, host_grads):
        self.done, self.host_img, self.host_grads = done, host_img, host_grads

    def wait(self):
        """Blocks until the step's image and gradients are in its host buffers."""
        self.done.synchronize()
        return self.host_img, self.host_grads


class HostPipeline:
    """Host-resident forward + backward steps queued back to back, with the
    copies of neighbouring steps overlapped (a training or serving loop whose
    scenes, upstream gradients, images and gradients live in pinned host memory).

    Two device slots (scene, upstream gradient, gradients) alternate between
    steps. Step i computes on the caller's stream while step i+1's scene and
    upstream gradient go up on an upload stream and step i-1's image and
    gradients come down on a download stream; each copy waits only for the
    step that last used its slot. The per-step copies are the same as
    HostStep's; they leave the critical path when steps follow one another.

    submit() queues one step (it returns once the forward's pair count is
    known, as render_forward does) and gives a handle whose wait() returns
    once that step's image and gradients are in its host buffers; finish()
    waits for every queued step. Host input buffers must stay unchanged, and
    host output buffers unread, until the step's wait() returns.
    """

    def __init__(self, like: DeviceScene, cams):
        self.cams = cams
        self.dev = like.means.device
        self.slots = []
        for _ in range(2):
            kw = {k: torch.empty_like(getattr(like, k)) for k in like.FLOAT_FIELDS + ("lobe_off",)}
            scene = DeviceScene(dtype_geom=like.dtype_geom, dtype_lobe=like.dtype_lobe,
                                dtype_sharp=like.dtype_sharp,
                                sh=None if like.sh is None else torch.empty_like(like.sh), **kw)
            self.slots.append(_Slot(scene, alloc_grads(scene)))
        self.up = torch.cuda.Stream(device=self.dev)
        self.down = torch.cuda.Stream(device=self.dev)
        self.i = 0

    def submit(self, host_scene: dict, host_d_img, host_img, host_grads: dict) -> PipelinedStep:
        slot = self.slots[self.i & 1]
        main = torch.cuda.current_stream(self.dev)
        fresh = slot.bwd_done is None
        if slot.d_img is None or slot.d_img.shape != host_d_img.shape:
            slot.d_img = torch.empty(host_d_img.shape, dtype=host_d_img.dtype, device=self.dev)
            fresh = True
        with torch.cuda.stream(self.up):
            if fresh:
                # memory allocated on the caller's stream may be a block that work
                # still queued there uses (the caching allocator orders it after
                # that work only on the caller's stream)
                self.up.wait_stream(main)
            else:                           # the slot's previous step has read its inputs
                self.up.wait_event(slot.bwd_done)
            for k, t in host_scene.items():
                getattr(slot.scene, k).copy_(t, non_blocking=True)
            slot.d_img.copy_(host_d_img, non_blocking=True)
            up_done = self.up.record_event()
        main.wait_event(up_done)
        out = render_forward(slot.scene, self.cams)
        if slot.down_done is not None:      # the slot's previous gradients are on the host
            main.wait_event(slot.down_done)
        render_backward(slot.scene, self.cams, out, slot.d_img, slot.grads)
        slot.bwd_done = main.record_event()
        with torch.cuda.stream(self.down):
            self.down.wait_event(slot.bwd_done)
            host_img.copy_(out.img.view(host_img.shape), non_blocking=True)
            for k, t in host_grads.items():
                t.copy_(slot.grads[k], non_blocking=True)
            slot.down_done = self.down.record_event()
        out.img.record_stream(self.down)
        self.i += 1
        return PipelinedStep(slot.down_done, host_img, host_grads)

    def finish(self):
        """Waits for every queued step."""
        for slot in self.slots:
            if slot.down_done is not None:
                slot.down_done.synchronize()

    @staticmethod
    def bytes_moved(host_scene: dict, host_d_img, host_img, host_grads: dict):
        """Host->device and device->host bytes of one step."""
        up = sum(t.numel() * t.element_size() for t in host_scene.values())
        up += host_d_img.numel() * host_d_img.element_size()
        down = host_img.numel() * host_img.element_size()
        down += sum(t.numel() * t.element_size() for t in host_grads.values())
        return up, down


class SGRasterize(torch.autograd.Function):
    """img, T_final, last = SGRasterize.apply(means, scales, quats, opac, gmask, c0,
    lobe_off, axis, sharp, amp, lmask, cams)

    Differentiable in every float input, the soft-pruning masks gmask (m_g) and
    lmask (m_l) included. T_final and last are saved for the backward, which
    therefore needs no re-sort; both are returned as non-differentiable outputs.
    """

    @staticmethod
    def forward(ctx, means, scales, quats, opac, gmask, c0, lobe_off, axis, sharp, amp, lmask, cams):
        dt = {torch.float32: _sg.SG_F32, torch.float16: _sg.SG_F16, torch.bfloat16: _sg.SG_BF16}
        scene = DeviceScene(means.contiguous(), scales.contiguous(), quats.contiguous(),
                            opac.contiguous(), gmask.contiguous(), c0.contiguous(),
                            lobe_off.contiguous(), axis.contiguous(), sharp.contiguous(),
                            amp.contiguous(), lmask.contiguous(), dtype_geom=dt[means.dtype],
                            dtype_lobe=dt[axis.dtype], dtype_sharp=dt[sharp.dtype])
        out = render_forward(scene, cams)
        ctx.scene = scene
        ctx.cams = cams
        ctx.sizes = out.sizes
        ctx.save_for_backward(out.ws, out.T_final, out.last)
        ctx.mark_non_differentiable(out.T_final, out.last)
        return out.img, out.T_final, out.last

    @staticmethod
    def backward(ctx, d_img, d_T, d_last):
        ws, T_final, last = ctx.saved_tensors
        fwd = ForwardOut(None, T_final, last, ws, ctx.sizes)
        grads = render_backward(ctx.scene, ctx.cams, fwd, d_img)
        sc = ctx.scene
        res = []
        for k in ("means", "scales", "quats", "opac", "gmask", "c0"):
            res.append(grads[k].to(getattr(sc, k).dtype))
        res.append(None)   # lobe_off
        for k in ("axis", "sharp", "amp", "lmask"):
            res.append(grads[k].to(getattr(sc, k).dtype))
        res.append(None)   # cams
        return tuple(res)


def rasterize(scene: DeviceScene, cams):
    """Autograd entry over a DeviceScene whose float tensors may require grad."""
    return SGRasterize.apply(scene.means, scene.scales, scene.quats, scene.opac, scene.gmask,
                             scene.c0, scene.lobe_off, scene.axis, scene.sharp, scene.amp,
                             scene.lmask, cams)


class BatchedRenderer:
    """Several scenes x cameras in one forward and one backward call.

    view_scene[v] is the scene of camera v. Outputs are flat and packed view
    after view: img [3 * sum HW] (each view [3][H][W]), T_final and last
    [sum HW]. The pair capacity is sized once (a probe forward records the
    need) with `headroom`; afterwards no call synchronises the host, so
    forward -> loss gradient -> backward can be captured in one CUDA graph.
    """

    def __init__(self, scenes, cams, view_scene, headroom=1.15, pair_capacity=None):
        self.scenes = list(scenes)
        self.cams = list(cams)
        self.view_scene = [int(v) for v in view_scene]
        dev = self.scenes[0].means.device
        self.device = dev
        self.npix = [int(c.width) * int(c.height) for c in self.cams]
        self.offsets = np.concatenate([[0], np.cumsum(self.npix)]).astype(np.int64)
        P = int(self.offsets[-1])
        self.img = torch.zeros(3 * P, device=dev)
        self.T_final = torch.ones(P, device=dev)
        self.last = torch.zeros(P, dtype=torch.int32, device=dev)
        self.d_img = torch.zeros(3 * P, device=dev)
        self.grads = [alloc_grads(sc) for sc in self.scenes]
        if pair_capacity is None:
            pair_capacity = self._probe_pairs()
        self.capacity = int(pair_capacity * headroom) + 4096
        self.sizes = _sg.sg_batched_workspace_query(self.scenes, self.cams, self.view_scene, self.capacity)
        self.ws = torch.empty(self.sizes["ws_bytes"], dtype=torch.uint8, device=dev)
        self.bwd = torch.empty(self.sizes["bwd_ws_bytes"], dtype=torch.uint8, device=dev)
        self.graph = None

    def _probe_pairs(self):
        q = _sg.sg_batched_workspace_query(self.scenes, self.cams, self.view_scene, 0)
        ws = torch.empty(q["ws_bytes"], dtype=torch.uint8, device=self.device)
        _sg.sg_render_batched_forward(self.scenes, self.cams, self.view_scene, ws, self.img,
                                      self.T_final, self.last)
        n, _ = _sg.sg_forward_status(ws)
        return n

    def view_image(self, v):
        o, n = int(self.offsets[v]), self.npix[v]
        c = self.cams[v]
        return self.img[3 * o:3 * (o + n)].view(3, c.height, c.width)

    def forward(self):
        _sg.sg_render_batched_forward(self.scenes, self.cams, self.view_scene, self.ws, self.img,
                                      self.T_final, self.last)
        return self.img

    def backward(self, d_img=None):
        if d_img is not None and d_img.data_ptr() != self.d_img.data_ptr():
            self.d_img.copy_(d_img.reshape(-1))
        _sg.sg_render_batched_backward(self.scenes, self.cams, self.view_scene, self.ws, self.T_final,
                                       self.last, self.d_img, self.bwd, self.grads)
        return self.grads

    def status(self):
        """(pairs the last forward needed, SG_OK or SG_ERR_CAPACITY); synchronises."""
        return _sg.sg_forward_status(self.ws)

    def step(self, loss_grad=None):
        """forward, d_img = loss_grad(img) (written in place), backward."""
        self.forward()
        if loss_grad is not None:
            loss_grad(self.img, self.d_img)
        self.backward()

    def autotune(self, loss_grad=None, reps=2):
        """Picks the blend shapes and batch sizes for this batch: every shape,
        then the batch sizes, each timed over eager steps with the library's
        stage events (the search of autotune.tune). Installs the choice (process
        wide) and returns it with the timings; capture afterwards."""
        from . import autotune
        return autotune.search(autotune.stage_measure(lambda: self.step(loss_grad), reps))

    def capture(self, loss_grad=None, warmup=2):
        """Captures step(loss_grad) in a CUDA graph; replay() runs it."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step(loss_grad)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step(loss_grad)
        return self.graph

    def replay(self):
        self.graph.replay()


def render_batched(scenes, cams, view_scene=None, **kw) -> BatchedRenderer:
    """Renders many scenes x cameras in one forward call: view_scene[v] is the
    scene of camera v (all scene 0 when omitted). Returns the BatchedRenderer
    holding the flat outputs (img, T_final, last, view_image(v)); its
    backward(d_img) gives every scene's gradients, summed over its views.
    Keyword arguments go to BatchedRenderer (headroom, pair_capacity)."""
    if view_scene is None:
        view_scene = [0] * len(cams)
    r = BatchedRenderer(scenes, cams, view_scene, **kw)
    r.forward()
    return r


def l1_loss_grad(renderer: BatchedRenderer, targets):
    """Upstream gradient of the per-view mean L1 loss against `targets`
    (flat, packed like img), summed over views: sign(img - target) / (3 H W)."""
    scale = torch.cat([torch.full((3 * n,), 1.0 / (3 * n), device=renderer.device)
                       for n in renderer.npix])

    def fn(img, out):
        torch.mul(torch.sign(img - targets), scale, out=out)
    return fn
