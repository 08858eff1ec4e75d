"""Failure detection on the GPU without a fault: the radix sorts' decoupled
look-back waits are bounded. With the bound set to one poll, a sort block that
finds a predecessor not yet published gives up at once and records
SG_ERR_TIMEOUT; the plain forward returns it and the batched form keeps it in
its device status. The outputs of such a call are unspecified, but every
access stays inside its buffers and the context stays usable: with the default
bound restored the next call renders what the oracle renders."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_07021_gb300 import render, sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

from parity_util import GpuView, check_image, gpu_view_lists

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _scene():
    rng = np.random.default_rng(880)
    scene = synth.make_scene(rng, 150_000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.6, masks="uniform")
    cam = synth.make_camera(640, 480, 600.0)
    return scene, cam


def test_sort_wait_bound_expires_and_is_reported():
    scene, cam = _scene()
    ds = DeviceScene.from_host(scene)
    ref = render.render_forward(ds, [cam])
    torch.cuda.synchronize()
    assert ref.sizes["n_pairs"] > 100_000          # hundreds of tile-sort blocks
    ws = torch.empty_like(ref.ws)
    img, T, last = torch.empty_like(ref.img), torch.empty_like(ref.T_final), torch.empty_like(ref.last)
    old = sgsplat.sg_get_tuning()
    plain, batched = [], []
    try:
        sgsplat.sg_set_tuning(sort_wait_polls=1)
        for _ in range(20):
            st, _ = sgsplat.sg_render_forward(ds, [cam], ws, img, T, last, raise_on_error=False)
            plain.append(st)
            if st == sgsplat.SG_ERR_TIMEOUT:
                assert "bounded device wait" in sgsplat.sg_last_error()
                break
        br = render.BatchedRenderer([ds], [cam], [0], pair_capacity=ref.sizes["n_pairs"])
        for _ in range(20):
            br.forward()
            _, st = br.status()
            batched.append(st)
            if st == sgsplat.SG_ERR_TIMEOUT:
                break
    finally:
        sgsplat.sg_set_tuning(**old)
    torch.cuda.synchronize()   # the context is still usable
    assert set(plain) <= {sgsplat.SG_OK, sgsplat.SG_ERR_TIMEOUT} and plain[-1] == sgsplat.SG_ERR_TIMEOUT
    assert set(batched) <= {sgsplat.SG_OK, sgsplat.SG_ERR_TIMEOUT} and batched[-1] == sgsplat.SG_ERR_TIMEOUT
    # default bound again: the same workspace renders what the oracle renders
    st, sizes = sgsplat.sg_render_forward(ds, [cam], ws, img, T, last, raise_on_error=False)
    assert st == sgsplat.SG_OK
    torch.cuda.synchronize()
    assert torch.equal(img, ref.img) and torch.equal(last, ref.last)
    sel = np.zeros(cam.n_tiles, bool)
    sel[np.random.default_rng(881).choice(cam.n_tiles, 24, replace=False)] = True
    res, _ = oracle.render(scene, [cam], tile_sel=[sel])
    fwd = render.ForwardOut(img, T, last, ws, sizes)
    gv = GpuView.plain(ds, [cam], fwd)
    m = np.repeat(np.repeat(sel.reshape(cam.tiles_y, cam.tiles_x), 16, 0), 16, 1)[:cam.height, :cam.width]
    check_image(img[0].cpu().numpy(), T[0].cpu().numpy(), last[0].cpu().numpy(), res[0], cam,
                gpu_view_lists(gv, [cam], 0), m)


def test_sort_wait_bound_rejects_negative():
    with pytest.raises(sgsplat.SGError):
        sgsplat.sg_set_tuning(sort_wait_polls=-1)
    sgsplat.sg_set_tuning()
    assert sgsplat.sg_get_tuning()["sort_wait_polls"] == 0
