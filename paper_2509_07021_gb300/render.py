"""Rendering front end: workspace management and the autograd Function.

PyTorch supplies device memory (every buffer is a torch tensor handed to the
C ABI as a pointer) and the current CUDA stream; the library does the rest.
"""
from __future__ import annotations

from dataclasses import dataclass

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


def render_forward(scene: DeviceScene, cams, stream=None) -> ForwardOut:
    device = scene.means.device
    img, T, last = _alloc_outputs(cams, device)
    key = _key(scene, cams)
    hint = _PAIR_HINT.get(key)
    if hint is None:
        hint = 8 * scene.n * len(cams)
    sizes = _sg.sg_workspace_query(scene, cams, int(hint * PAIR_HEADROOM) + 1024)
    ws = torch.empty(sizes["ws_bytes"], dtype=torch.uint8, device=device)
    st, out = _sg.sg_render_forward(scene, cams, ws, img, T, last, stream, raise_on_error=False)
    if st == _sg.SG_ERR_CAPACITY:
        sizes = _sg.sg_workspace_query(scene, cams, int(out["n_pairs"] * PAIR_HEADROOM) + 1024)
        ws = torch.empty(sizes["ws_bytes"], dtype=torch.uint8, device=device)
        st, out = _sg.sg_render_forward(scene, cams, ws, img, T, last, stream, raise_on_error=False)
    if st != _sg.SG_OK:
        raise SGError(st, _sg.sg_last_error())
    _PAIR_HINT[key] = out["n_pairs"]
    return ForwardOut(img, T, last, ws, out)


def alloc_grads(scene: DeviceScene):
    return {k: torch.empty(getattr(scene, k).shape, dtype=torch.float32, device=scene.means.device)
            for k in DeviceScene.FLOAT_FIELDS}


def render_backward(scene: DeviceScene, cams, fwd: ForwardOut, d_img, grads=None, stream=None):
    """Gradients of sum(d_img * img) for every float input (binary32 tensors)."""
    if grads is None:
        grads = alloc_grads(scene)
    bwd = torch.empty(fwd.sizes["bwd_ws_bytes"], dtype=torch.uint8, device=scene.means.device)
    _sg.sg_render_backward(scene, cams, fwd.ws, fwd.T_final, fwd.last, d_img.contiguous(), bwd,
                           grads, stream)
    return grads


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
