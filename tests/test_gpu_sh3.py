"""The degree-3 SH colour model (the 3DGS baseline representation) on the CUDA
path vs the FP64 oracle, through the C ABI: same tolerances as the SG model
(tile lists bit exact, image max abs error <= 2e-4, gradients relative L2 <= 1e-3
per tensor, the SH coefficients included)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_07021_gb300 import render, sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

from test_gpu_parity import run_parity

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sgsplat.lib()
    oracle.lib()


def _sh_scene(seed, n, **kw):
    rng = np.random.default_rng(seed)
    sg = synth.make_scene(rng, n, lobes=0, **kw)
    return synth.with_sh3_colour(sg, rng)


def test_sh3_config0_shape_forward_backward():
    """1,000 Gaussians at 128x128 (the small SG workload's geometry) with SH3 colour."""
    sg, cams = synth.config0()
    scene = synth.with_sh3_colour(sg, np.random.default_rng(90))
    rep, grep = run_parity(scene, cams, seed=5)
    assert rep[0]["max_abs_err"] <= 2e-4
    assert grep["sh"] <= 1e-3


def test_sh3_ragged_multi_view():
    """Ragged image size, soft masks, background, two views summed into the
    SH gradients."""
    scene = _sh_scene(91, 5000, means="cube", cube_side=1.4, masks="uniform")
    cams = [synth.make_camera(100, 70, 90.0, bg=(0.2, 0.4, 0.1)),
            synth.make_camera(100, 70, 90.0, bg=(0.2, 0.4, 0.1),
                              viewmat=synth.look_at((0.7, -0.3, 0.4), (0.0, 0.0, 4.0)))]
    rep, grep = run_parity(scene, cams, seed=6)
    assert max(r["max_abs_err"] for r in rep) <= 2e-4


def test_sh3_invisible_gaussians_get_zero_sh_grads():
    """Gaussians behind the camera: their SH gradients are written as zeros."""
    scene = _sh_scene(92, 300, means="cube")
    scene.means[2, :100] = -5.0
    ds = DeviceScene.from_host(scene)
    cams = [synth.make_camera(48, 48, 60.0)]
    out = render.render_forward(ds, cams)
    grads = render.alloc_grads(ds)
    for g in grads.values():
        g.fill_(float("nan"))
    d = torch.ones(1, 3, 48, 48, device="cuda")
    render.render_backward(ds, cams, out, d, grads=grads)
    torch.cuda.synchronize()
    sh = grads["sh"].cpu().numpy()
    assert np.all(sh[:, :, :100] == 0.0)
    assert np.all(np.isfinite(sh))


def test_sh3_rejects_half_storage_and_lobes():
    scene = _sh_scene(93, 64, means="cube")
    cams = [synth.make_camera(32, 32, 40.0)]
    ds = DeviceScene.from_host(scene, storage="f16")
    with pytest.raises(sgsplat.SGError, match="SH3"):
        render.render_forward(ds, cams)
    rng = np.random.default_rng(94)
    with_lobes = synth.make_scene(rng, 64, lobes=1, means="cube")
    with_lobes.sh = scene.sh
    ds = DeviceScene.from_host(with_lobes)
    assert ds.color_model == sgsplat.SG_COLOR_SH3 and ds.n_lobes == 64
    with pytest.raises(sgsplat.SGError, match="SH3"):
        render.render_forward(ds, cams)
