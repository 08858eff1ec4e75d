"""The backward entry point that allocates nothing.

Some callers cannot allocate device memory while they render (a frame loop or
a serving process that reserves its GPU memory up front, code that must not
synchronise the device through cudaMalloc). sg_render_backward_noalloc takes
its scratch from a static array inside the library instead; its gradients
must match sg_render_backward's, call after call.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2509_07021_gb300 import render, sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

from parity_util import GRAD_TOL, rel_l2

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _scene_and_grad(seed=0, n=3000):
    rng = np.random.default_rng(900 + seed)
    scene = synth.make_scene(rng, n, lobes=synth.LOBE_MIX, means="cube", cube_side=1.2,
                             masks="uniform")
    cam = synth.make_camera(96, 72, 100.0, bg=(0.1, 0.2, 0.3))
    d_img = torch.from_numpy(rng.normal(0, 0.01, (1, 3, 72, 96)).astype(np.float32)).cuda()
    return scene, [cam], d_img


def test_noalloc_backward_matches_backward_twice():
    scene, cams, d_img = _scene_and_grad()
    ds = DeviceScene.from_host(scene)
    out = render.render_forward(ds, cams)
    ref = render.render_backward(ds, cams, out, d_img)
    torch.cuda.synchronize()
    assert out.sizes["bwd_ws_bytes"] <= sgsplat.SG_NOALLOC_SCRATCH_BYTES
    for _ in range(2):
        got = render.alloc_grads(ds)
        for v in got.values():
            v.fill_(float("nan"))   # every gradient must be overwritten
        sgsplat.sg_render_backward_noalloc(ds, cams, out.ws, out.T_final, out.last, d_img, got)
        torch.cuda.synchronize()
        for k, r in ref.items():
            a = got[k].cpu().numpy().astype(np.float64)
            b = r.cpu().numpy().astype(np.float64)
            assert np.isfinite(a).all(), k
            assert rel_l2(a, b) <= GRAD_TOL, k


def test_noalloc_backward_rejects_oversized_calls():
    """Beyond the static scratch the call fails with SG_ERR_WORKSPACE before any device work."""
    n = sgsplat.SG_NOALLOC_SCRATCH_BYTES // 36 + 1000
    f = np.float32
    scene = synth.Scene(means=np.zeros((3, n), f), scales=np.ones((3, n), f),
                        quats=np.ones((4, n), f), opac=np.ones(n, f), gmask=np.ones(n, f),
                        c0=np.zeros((3, n), f), lobe_off=np.zeros(n + 1, np.int32),
                        axis=np.zeros((3, 0), f), sharp=np.zeros(0, f), amp=np.zeros((3, 0), f),
                        lmask=np.zeros(0, f))
    ds = DeviceScene.from_host(scene)
    cams = [synth.make_camera(32, 32, 40.0)]
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    img = torch.zeros(1, 3, 32, 32, device="cuda")
    T = torch.ones(1, 32, 32, device="cuda")
    last = torch.zeros(1, 32, 32, dtype=torch.int32, device="cuda")
    grads = render.alloc_grads(ds)
    st = sgsplat.sg_render_backward_noalloc(ds, cams, ws, T, last, img, grads,
                                            raise_on_error=False)
    assert st == sgsplat.SG_ERR_WORKSPACE
    assert "static scratch" in sgsplat.sg_last_error()
