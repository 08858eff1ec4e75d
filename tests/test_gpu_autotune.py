"""sg_autotune (C ABI): times all eight blend shapes, then the batch sizes, on
the caller's buffers, installs the fastest forward and backward choice, and
leaves correct results."""
import numpy as np
import pytest
import torch

from paper_2509_07021_gb300 import render, sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_autotune_installs_a_valid_choice_and_keeps_results():
    sgsplat.lib()
    old = sgsplat.sg_get_tuning()
    try:
        rng = np.random.default_rng(77)
        scene = synth.make_scene(rng, 3000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.4, masks="uniform")
        cams = [synth.make_camera(96, 64, 80.0, bg=(0.1, 0.2, 0.3))]
        ds = DeviceScene.from_host(scene)
        sgsplat.sg_set_tuning()
        ref = render.render_forward(ds, cams)
        d_img = torch.from_numpy(rng.normal(0, 0.01, (1, 3, 64, 96)).astype(np.float32)).cuda()
        g_ref = render.render_backward(ds, cams, ref, d_img)
        img = torch.empty_like(ref.img)
        T = torch.empty_like(ref.T_final)
        last = torch.empty_like(ref.last)
        bwd = torch.empty(ref.sizes["bwd_ws_bytes"], dtype=torch.uint8, device="cuda")
        grads = render.alloc_grads(ds)
        got = sgsplat.sg_autotune(ds, cams, ref.ws, img, T, last, d_img, bwd, grads, reps=2)
        torch.cuda.synchronize()
        t = sgsplat.sg_get_tuning()
        for k in ("fwd_pixels_per_thread", "bwd_pixels_per_thread", "fwd_persistent", "bwd_persistent",
                  "fwd_batch", "bwd_batch"):
            assert t[k] == got[k]
        assert t["fwd_pixels_per_thread"] in (1, 2, 4, 8) and t["bwd_persistent"] in (0, 1)
        assert t["fwd_batch"] in (32, 64, 128) and t["bwd_batch"] in (32, 64)
        assert len(got["ms"]) == 8 and all(v["fwd_call"] > 0 and v["bwd_call"] > 0 for v in got["ms"].values())
        fastest_f = min(got["ms"].values(), key=lambda v: v["fwd_call"])["fwd_call"]
        name = f"p{t['fwd_pixels_per_thread']}" + ("_persistent" if t["fwd_persistent"] else "")
        assert got["ms"][name]["fwd_call"] == fastest_f
        assert torch.equal(img, ref.img) and torch.equal(T, ref.T_final) and torch.equal(last, ref.last)
        for k, v in g_ref.items():
            if v.numel() and float(v.norm()) > 0:
                assert float((grads[k] - v).norm() / v.norm()) <= 1e-5, k
    finally:
        sgsplat.sg_set_tuning(**old)


def test_autotune_rejects_bad_reps():
    sgsplat.lib()
    scene, cams = synth.config0()
    ds = DeviceScene.from_host(scene)
    out = render.render_forward(ds, cams)
    bwd = torch.empty(out.sizes["bwd_ws_bytes"], dtype=torch.uint8, device="cuda")
    grads = render.alloc_grads(ds)
    d = torch.zeros_like(out.img)
    with pytest.raises(sgsplat.SGError):
        sgsplat.sg_autotune(ds, cams, out.ws, out.img, out.T_final, out.last, d, bwd, grads, reps=0)


def test_batched_autotune_picks_valid_shapes_and_keeps_results():
    """BatchedRenderer.autotune runs the same search over the batch (every shape,
    then the batch sizes), installs the fastest choice, and the captured step
    reproduces the images of the default shapes."""
    sgsplat.lib()
    old = sgsplat.sg_get_tuning()
    try:
        rng = np.random.default_rng(78)
        scenes = [DeviceScene.from_host(synth.make_scene(rng, n, lobes=synth.LOBE_MIX, means="cube",
                                                         cube_side=1.4, masks="uniform")) for n in (2000, 700)]
        cams = [synth.make_camera(96, 64, 80.0), synth.make_camera(48, 80, 60.0), synth.make_camera(64, 64, 70.0)]
        view_scene = [0, 1, 1]
        sgsplat.sg_set_tuning()
        br = render.BatchedRenderer(scenes, cams, view_scene)
        br.forward()
        ref = br.img.clone()
        got = br.autotune(reps=1)
        t = sgsplat.sg_get_tuning()
        for k in ("fwd_pixels_per_thread", "bwd_pixels_per_thread", "fwd_persistent", "bwd_persistent",
                  "fwd_batch", "bwd_batch"):
            assert t[k] == got[k]
        assert t["fwd_batch"] in (32, 64, 128) and t["bwd_batch"] in (32, 64)
        assert len(got["ms"]) == 8 and len(got["batch_ms"]) == 3
        fastest_b = min(v["blend_bwd"] for v in got["ms"].values())
        name = f"p{t['bwd_pixels_per_thread']}" + ("_persistent" if t["bwd_persistent"] else "")
        assert got["ms"][name]["blend_bwd"] == fastest_b
        br.capture()
        br.replay()
        torch.cuda.synchronize()
        assert torch.equal(br.img, ref)
    finally:
        sgsplat.sg_set_tuning(**old)
