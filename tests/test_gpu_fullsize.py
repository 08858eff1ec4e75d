"""Parity at the full sizes the benchmark runs, in its launch configuration
(the library's default blend shapes), on sampled tiles the oracle can afford:

* the headline scene: 1M Gaussians, lobes 0-4, soft masks, one 1920x1080 view
  (plain forward + backward);
* the batched workload: 8 uneven scenes (50k .. 2M Gaussians) x 4 cameras at
  mixed resolutions in one batched call, two of its views checked;
* the stress workload: 6M Gaussians, 60 % / 50 % exact-zero masks, a packed
  cluster, 16 views in one batched call, one view checked.

Over the whole frame of every checked view: the tile lists are ordered
sub-lists of the oracle's 3-sigma-rectangle lists, every pair left out is
proven unreachable in FP64, and lists, tiles_touched and ranges equal the
library's binning rule bit for bit. Images, T, last and gradients on the
sampled tiles (the upstream gradient is zero elsewhere, so the oracle's
gradients are exact for it)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_07021_gb300 import render, sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

from parity_util import (GpuView, check_decisions, check_grads, check_image, gpu_view_lists, masked_dimg,
                         pixel_mask_of_tiles, unpack_views)

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(autouse=True)
def _default_shapes():
    sgsplat.lib()
    oracle.lib()
    old = sgsplat.sg_get_tuning()
    sgsplat.sg_set_tuning()
    yield
    sgsplat.sg_set_tuning(**old)


def _sample(cam, n, seed):
    sel = np.zeros(cam.n_tiles, bool)
    sel[np.random.default_rng(seed).choice(cam.n_tiles, n, replace=False)] = True
    sel[cam.n_tiles - 1] = True   # the ragged corner tile
    return sel


def test_headline_scene_1m_1080p():
    scene, cams, _ = synth.config3()
    cam = cams[0]
    ds = DeviceScene.from_host(scene)
    out = render.render_forward(ds, cams)
    torch.cuda.synchronize()
    sel = _sample(cam, 32, 31)
    results, _ = oracle.render(scene, cams, tile_sel=[sel])
    gv = GpuView.plain(ds, cams, out)
    check_decisions(gv, cams, [(0, scene, results[0])])
    rep = check_image(unpack_views(out.img, cams, 3)[0], unpack_views(out.T_final, cams, 1)[0],
                      unpack_views(out.last, cams, 1)[0], results[0], cam, gpu_view_lists(gv, cams, 0),
                      pixel_mask_of_tiles(cam, sel))
    assert rep["ambiguous"] <= 0.01 * rep["pixels"]
    dimgs = masked_dimg(np.random.default_rng(32), cams, results, [sel])
    _, g_orc = oracle.render(scene, cams, dimgs=dimgs, tile_sel=[sel])
    g = render.render_backward(ds, cams, out, torch.from_numpy(np.stack(dimgs)).cuda())
    torch.cuda.synchronize()
    check_grads(g, g_orc)


def _batched_views(scenes, cams, view_scene, checks, seed):
    """One batched forward + backward over all views; the views in `checks`
    are compared with the oracle on sampled tiles (upstream gradient zero on
    every other view and tile)."""
    dss = [DeviceScene.from_host(s) for s in scenes]
    br = render.BatchedRenderer(dss, cams, view_scene)
    br.forward()
    n, st = br.status()
    assert st == sgsplat.SG_OK and n <= br.capacity
    torch.cuda.synchronize()
    d_all = np.zeros(br.d_img.numel(), np.float32)
    oracle_grads = {}
    gv = GpuView.batched(br)
    for v, n_tiles in checks:
        cam, s = cams[v], view_scene[v]
        sel = _sample(cam, n_tiles, seed + v)
        res, _ = oracle.render(scenes[s], [cam], tile_sel=[sel])
        check_decisions(gv, cams, [(v, scenes[s], res[0])])
        o, npx = int(br.offsets[v]), br.npix[v]
        img = br.img[3 * o:3 * (o + npx)].view(3, cam.height, cam.width).cpu().numpy()
        T = br.T_final[o:o + npx].view(cam.height, cam.width).cpu().numpy()
        last = br.last[o:o + npx].view(cam.height, cam.width).cpu().numpy()
        check_image(img, T, last, res[0], cam, gpu_view_lists(gv, cams, v), pixel_mask_of_tiles(cam, sel))
        dimg = masked_dimg(np.random.default_rng(seed + 100 + v), [cam], res, [sel])[0]
        d_all[3 * o:3 * (o + npx)] = dimg.reshape(-1)
        _, g = oracle.render(scenes[s], [cam], dimgs=[dimg], tile_sel=[sel])
        oracle_grads[s] = g if s not in oracle_grads else {k: oracle_grads[s][k] + g[k] for k in g}
    br.backward(torch.from_numpy(d_all).cuda())
    torch.cuda.synchronize()
    for s, g in oracle_grads.items():
        check_grads(br.grads[s], g)


def test_batched_workload_two_views():
    scenes, cams_per, _ = synth.config2()
    cams = [c for cs in cams_per for c in cs]
    view_scene = [s for s, cs in enumerate(cams_per) for _ in cs]
    # the largest scene at 1920x1080 and the smallest at 800x800
    _batched_views(scenes, cams, view_scene, [(4 * 7 + 3, 24), (0, 24)], seed=40)


def test_stress_workload_one_view():
    scene, cams, _ = synth.config4()
    _batched_views([scene], cams, [0] * len(cams), [(5, 16)], seed=50)
