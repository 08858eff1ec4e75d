"""render.HostStep (pinned host inputs and outputs, copies overlapped on a
second stream) returns exactly what the device-resident forward + backward
returns."""
import numpy as np
import pytest
import torch

from paper_2509_07021_gb300 import render, sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_host_step_matches_device_step():
    sgsplat.lib()
    rng = np.random.default_rng(71)
    scene = synth.make_scene(rng, 4000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.4, masks="uniform")
    cams = [synth.make_camera(100, 70, 90.0, bg=(0.2, 0.4, 0.1))]
    d_img = rng.normal(0, 0.01, (1, 3, 70, 100)).astype(np.float32)

    ref = DeviceScene.from_host(scene)
    out = render.render_forward(ref, cams)
    g_ref = render.render_backward(ref, cams, out, torch.from_numpy(d_img).cuda())
    torch.cuda.synchronize()

    ds = DeviceScene.from_host(scene)
    fields = list(DeviceScene.FLOAT_FIELDS) + ["lobe_off"]
    host_in = {k: getattr(ds, k).cpu().pin_memory() for k in fields}
    for k in DeviceScene.FLOAT_FIELDS:          # the step must upload the inputs itself
        getattr(ds, k).zero_()
    host_dimg = torch.from_numpy(d_img).pin_memory()
    host_img = torch.empty((1, 3, 70, 100)).pin_memory()
    host_grads = {k: torch.empty(v.shape).pin_memory() for k, v in g_ref.items()}
    step = render.HostStep(ds, cams, host_in, host_dimg, host_img, host_grads)
    for _ in range(2):
        img, grads = step()
        assert torch.equal(img, out.img.cpu())
        for k, v in g_ref.items():   # atomics sum in any order: relative L2, not bits
            a, b = grads[k].numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
            nb = np.linalg.norm(b)
            assert (np.linalg.norm(a - b) / nb if nb else np.abs(a).max()) <= 1e-5, k
    up, down = step.bytes_moved()
    assert up == sum(t.numel() * t.element_size() for t in host_in.values()) + host_dimg.numel() * 4
    assert down == host_img.numel() * 4 + sum(t.numel() * 4 for t in host_grads.values())
