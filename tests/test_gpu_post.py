"""Post-processing on the GPU (Sec. 3.3.3) vs the oracle: kept Gaussians and
lobes bit exact, compensated colour within binary32 rounding."""
import numpy as np
import pytest
import torch

from oracle import post
from paper_2509_07021_gb300 import sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("n,tau_o", [(5000, 0.1), (60000, 0.25), (1, 0.0), (300, 2.0)])
def test_postprocess_matches_oracle(n, tau_o):
    rng = np.random.default_rng(n)
    scene = synth.make_scene(rng, n, lobes=synth.LOBE_MIX, masks="uniform")
    scene.sharp[::3] = rng.uniform(-0.5, 1.5, scene.sharp[::3].size).astype(np.float32)
    scene.sharp[::17] = 0.0
    ds = DeviceScene.from_host(scene)
    out = sgsplat.sg_postprocess(ds, tau_o, 1.0)
    torch.cuda.synchronize()
    gid, lid, off, c0 = post.postprocess(scene, tau_o, 1.0)
    assert out.n == len(gid) and out.n_lobes == len(lid)
    np.testing.assert_array_equal(out.lobe_off.cpu().numpy(), off)
    for k in ("means", "scales", "quats"):
        np.testing.assert_array_equal(getattr(out, k).cpu().numpy(), getattr(scene, k)[:, gid])
    for k in ("opac", "gmask"):
        np.testing.assert_array_equal(getattr(out, k).cpu().numpy(), getattr(scene, k)[gid])
    for k in ("axis", "amp"):
        np.testing.assert_array_equal(getattr(out, k).cpu().numpy(), getattr(scene, k)[:, lid])
    for k in ("sharp", "lmask"):
        np.testing.assert_array_equal(getattr(out, k).cpu().numpy(), getattr(scene, k)[lid])
    np.testing.assert_allclose(out.c0.cpu().numpy(), c0, rtol=2e-6, atol=2e-6)


def test_postprocessed_scene_renders():
    """The compacted scene is a valid input of the renderer."""
    from paper_2509_07021_gb300 import render
    rng = np.random.default_rng(3)
    scene = synth.make_scene(rng, 3000, lobes=synth.LOBE_MIX, means="cube", masks="uniform")
    ds = sgsplat.sg_postprocess(DeviceScene.from_host(scene), 0.05, 1.0)
    out = render.render_forward(ds, [synth.make_camera(64, 64, 80.0)])
    torch.cuda.synchronize()
    assert torch.isfinite(out.img).all() and out.sizes["n_pairs"] > 0
