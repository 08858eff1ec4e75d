"""Batched form vs the FP64 oracle: several scenes of uneven size, cameras at
mixed resolutions, one forward and one backward call, graph capture, and the
persistent (work-queue) blend."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_07021_gb300 import render, sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

from parity_util import GpuView, check_decisions, check_grads, check_image, gpu_view_lists, masked_dimg
from test_gpu_parity import check_importance, unambiguous_gaussians

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _batch(seed=0):
    rng = np.random.default_rng(700 + seed)
    scenes = [synth.make_scene(rng, n, lobes=synth.LOBE_MIX, means="cube", cube_side=1.3,
                               masks="uniform") for n in (2500, 700, 4100)]
    cams = [synth.make_camera(64, 48, 60.0),
            synth.make_camera(40, 40, 45.0, viewmat=synth.look_at((0.4, 0.2, 0.1), (0, 0, 4.0))),
            synth.make_camera(33, 21, 30.0, bg=(0.2, 0.3, 0.4)),
            synth.make_camera(80, 50, 70.0, viewmat=synth.look_at((-0.5, 0.0, 0.3), (0, 0, 4.0))),
            synth.make_camera(16, 16, 20.0)]
    view_scene = [0, 1, 0, 2, 1]
    return scenes, cams, view_scene


def _flat_views(t, cams, ch):
    a = t.detach().cpu().numpy()
    out, o = [], 0
    for c in cams:
        n = c.width * c.height * ch
        x = a[o:o + n]
        out.append(x.reshape(3, c.height, c.width) if ch == 3 else x.reshape(c.height, c.width))
        o += n
    return out


def _check_batched(br, scenes, cams, view_scene, seed):
    imgs = _flat_views(br.img, cams, 3)
    Ts = _flat_views(br.T_final, cams, 1)
    lasts = _flat_views(br.last, cams, 1)
    results = []
    gv = GpuView.batched(br)
    for v, cam in enumerate(cams):
        res, _ = oracle.render(scenes[view_scene[v]], [cam])
        results.append(res[0])
        check_decisions(gv, cams, [(v, scenes[view_scene[v]], res[0])])
        check_image(imgs[v], Ts[v], lasts[v], res[0], cam, gpu_view_lists(gv, cams, v))
    rng = np.random.default_rng(seed)
    dimgs = masked_dimg(rng, cams, results)
    br.backward(torch.from_numpy(np.concatenate([d.reshape(-1) for d in dimgs])).cuda())
    torch.cuda.synchronize()
    for s, scene in enumerate(scenes):
        vs = [v for v in range(len(cams)) if view_scene[v] == s]
        _, g = oracle.render(scene, [cams[v] for v in vs], dimgs=[dimgs[v] for v in vs])
        check_grads(br.grads[s], g)


@pytest.mark.parametrize("persistent", [0, 1])
def test_batched_multi_scene_parity(persistent):
    scenes, cams, view_scene = _batch()
    ds = [DeviceScene.from_host(s) for s in scenes]
    old = sgsplat.sg_get_tuning()
    sgsplat.sg_set_tuning(fwd_persistent=persistent, bwd_persistent=persistent)
    try:
        br = render.BatchedRenderer(ds, cams, view_scene)
        br.forward()
        n, st = br.status()
        assert st == sgsplat.SG_OK and 0 < n <= br.capacity
        _check_batched(br, scenes, cams, view_scene, seed=persistent)
    finally:
        sgsplat.sg_set_tuning(**old)


def test_render_batched_function():
    """render.render_batched: one call renders every view; the same outputs as a
    BatchedRenderer driven by hand."""
    scenes, cams, view_scene = _batch(5)
    ds = [DeviceScene.from_host(s) for s in scenes]
    r = render.render_batched(ds, cams, view_scene)
    br = render.BatchedRenderer(ds, cams, view_scene)
    br.forward()
    torch.cuda.synchronize()
    assert torch.equal(r.img, br.img) and torch.equal(r.T_final, br.T_final) and torch.equal(r.last, br.last)
    gv = GpuView.batched(r)
    for v, cam in enumerate(cams):
        res, _ = oracle.render(scenes[view_scene[v]], [cam])
        check_image(*(_flat_views(t, cams, ch)[v] for t, ch in ((r.img, 3), (r.T_final, 1), (r.last, 1))),
                    res[0], cam, gpu_view_lists(gv, cams, v))


def test_persistent_plain_form():
    scenes, cams, _ = _batch(1)
    old = sgsplat.sg_get_tuning()
    sgsplat.sg_set_tuning(fwd_persistent=1, bwd_persistent=1)
    try:
        from test_gpu_parity import run_parity
        run_parity(scenes[2], [cams[3]], seed=5)
    finally:
        sgsplat.sg_set_tuning(**old)


def test_batched_capacity_overflow_is_reported():
    scenes, cams, view_scene = _batch(2)
    ds = [DeviceScene.from_host(s) for s in scenes]
    br = render.BatchedRenderer(ds, cams, view_scene, pair_capacity=10, headroom=1.0)
    assert br.capacity == 10 + 4096
    br.forward()
    need, st = br.status()
    big = render.BatchedRenderer(ds, cams, view_scene)
    big.forward()
    need2, st2 = big.status()
    assert st2 == sgsplat.SG_OK
    if need2 > br.capacity:
        assert st == sgsplat.SG_ERR_CAPACITY and need == need2
        # nothing was binned: every pixel shows the background
        assert torch.all(br.T_final == 1)
    else:
        assert st == sgsplat.SG_OK


def test_graph_replay_matches_eager():
    scenes, cams, view_scene = _batch(3)
    ds = [DeviceScene.from_host(s) for s in scenes]
    br = render.BatchedRenderer(ds, cams, view_scene)
    targets = torch.rand(br.img.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    lg = render.l1_loss_grad(br, targets)
    br.step(lg)
    torch.cuda.synchronize()
    eager_img = br.img.clone()
    eager = [{k: v.clone() for k, v in g.items()} for g in br.grads]
    br.capture(lg)
    for g in br.grads:
        for v in g.values():
            v.zero_()
    br.img.zero_()
    br.replay()
    br.replay()
    torch.cuda.synchronize()
    assert torch.equal(br.img, eager_img)
    for g, e in zip(br.grads, eager):
        for k in g:
            a, b = g[k].double(), e[k].double()
            # atomics make the summation order differ between runs
            assert torch.linalg.norm(a - b) <= 1e-5 * torch.linalg.norm(b) + 1e-12, k
    n, st = br.status()
    assert st == sgsplat.SG_OK


def test_batched_importance_per_scene():
    scenes, cams, view_scene = _batch(4)
    ds = [DeviceScene.from_host(s) for s in scenes]
    br = render.BatchedRenderer(ds, cams, view_scene)
    imps = [torch.zeros(d.n, device="cuda") for d in ds]
    sgsplat.sg_render_batched_forward(ds, cams, view_scene, br.ws, br.img, br.T_final, br.last,
                                      importance=imps)
    torch.cuda.synchronize()
    for s, scene in enumerate(scenes):
        vs = [v for v in range(len(cams)) if view_scene[v] == s]
        results, _ = oracle.render(scene, [cams[v] for v in vs])
        expect = sum(r.importance for r in results)
        got = imps[s].cpu().numpy().astype(np.float64)
        check_importance(got, expect, unambiguous_gaussians(results, scene.n))


@pytest.mark.parametrize("sizes", [[(16, 16)], [(20, 12)]])
def test_batched_one_or_two_tiles(sizes):
    """A frame of one tile (the tile sort has no pass: its ranges come from the
    pair count alone) and of two tiles (one pass) through the batched form."""
    rng = np.random.default_rng(720 + len(sizes))
    scene = synth.make_scene(rng, 600, lobes=synth.LOBE_MIX, means="cube", cube_side=1.3, masks="uniform")
    cams = [synth.make_camera(w, h, 20.0) for w, h in sizes]
    ds = [DeviceScene.from_host(scene)]
    br = render.BatchedRenderer(ds, cams, [0] * len(cams))
    br.forward()
    n, st = br.status()
    assert st == sgsplat.SG_OK and 0 < n <= br.capacity
    _check_batched(br, [scene], cams, [0] * len(cams), seed=7)


def test_batched_scene_without_views():
    """Two scenes and one view that sees only the smaller one: the larger scene
    has no view, so its gradients are zero, and the seen scene's gradients are
    the one-view oracle's (the adjoint's one-view path tests the view's scene)."""
    rng = np.random.default_rng(730)
    scenes = [synth.make_scene(rng, n, lobes=synth.LOBE_MIX, means="cube", cube_side=1.3, masks="uniform")
              for n in (4100, 700)]
    cams = [synth.make_camera(40, 40, 45.0)]
    view_scene = [1]
    ds = [DeviceScene.from_host(s) for s in scenes]
    br = render.BatchedRenderer(ds, cams, view_scene)
    br.forward()
    n, st = br.status()
    assert st == sgsplat.SG_OK and 0 < n <= br.capacity
    res, _ = oracle.render(scenes[1], cams)
    img, T, last = (_flat_views(t, cams, ch)[0] for t, ch in ((br.img, 3), (br.T_final, 1), (br.last, 1)))
    gv = GpuView.batched(br)
    check_decisions(gv, cams, [(0, scenes[1], res[0])])
    check_image(img, T, last, res[0], cams[0], gpu_view_lists(gv, cams, 0))
    dimgs = masked_dimg(np.random.default_rng(731), cams, res)
    for g in br.grads[0].values():
        g.fill_(7.0)   # gradients are overwritten, never accumulated
    br.backward(torch.from_numpy(dimgs[0].reshape(-1)).cuda())
    torch.cuda.synchronize()
    for k, v in br.grads[0].items():
        assert torch.count_nonzero(v) == 0, k
    _, g = oracle.render(scenes[1], cams, dimgs=dimgs)
    check_grads(br.grads[1], g)
