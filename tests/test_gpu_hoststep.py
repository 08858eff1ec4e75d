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


def test_host_pipeline_matches_device_steps():
    """Five queued steps alternating between two scenes, each with its own
    upstream gradient and host output buffers: every step returns what its own
    device-resident forward + backward returns (the two device slots never mix
    steps up)."""
    sgsplat.lib()
    rng = np.random.default_rng(72)
    a = synth.make_scene(rng, 3000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.4, masks="uniform")
    b = a.copy()   # same shapes, other values
    b.means += rng.normal(0, 0.05, b.means.shape).astype(np.float32)
    b.c0 = rng.uniform(0, 1, b.c0.shape).astype(np.float32)
    b.amp = rng.normal(0, 0.3, b.amp.shape).astype(np.float32)
    cams = [synth.make_camera(90, 60, 80.0, bg=(0.1, 0.2, 0.3))]
    fields = list(DeviceScene.FLOAT_FIELDS) + ["lobe_off"]
    steps = []
    for i in range(5):
        sc = (a, b)[i % 2]
        ds = DeviceScene.from_host(sc)
        d_img = rng.normal(0, 0.01, (1, 3, 60, 90)).astype(np.float32)
        out = render.render_forward(ds, cams)
        g = render.render_backward(ds, cams, out, torch.from_numpy(d_img).cuda())
        host_in = {k: getattr(ds, k).cpu().pin_memory() for k in fields}
        steps.append(dict(ref_img=out.img.cpu(), ref_g={k: v.cpu() for k, v in g.items()},
                          host_in=host_in, host_dimg=torch.from_numpy(d_img).pin_memory(),
                          host_img=torch.full((1, 3, 60, 90), float("nan")).pin_memory(),
                          host_grads={k: torch.full(v.shape, float("nan")).pin_memory() for k, v in g.items()}))
    torch.cuda.synchronize()
    pipe = render.HostPipeline(DeviceScene.from_host(a), cams)
    handles = [pipe.submit(s["host_in"], s["host_dimg"], s["host_img"], s["host_grads"]) for s in steps]
    pipe.finish()
    for s, h in zip(steps, handles):
        img, grads = h.wait()
        assert torch.equal(img, s["ref_img"])
        for k, v in s["ref_g"].items():
            x, y = grads[k].numpy().astype(np.float64), v.numpy().astype(np.float64)
            ny = np.linalg.norm(y)
            assert (np.linalg.norm(x - y) / ny if ny else np.abs(x).max()) <= 1e-5, k
    up, down = render.HostPipeline.bytes_moved(steps[0]["host_in"], steps[0]["host_dimg"],
                                               steps[0]["host_img"], steps[0]["host_grads"])
    assert up == sum(t.numel() * t.element_size() for t in steps[0]["host_in"].values()) + 3 * 60 * 90 * 4
    assert down == 3 * 60 * 90 * 4 + sum(t.numel() * 4 for t in steps[0]["host_grads"].values())
