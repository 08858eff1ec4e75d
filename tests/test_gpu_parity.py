"""CUDA path vs the FP64 oracle, through the C ABI.

Tile decisions bit exact; every tile list an ordered sub-list of the oracle's
3-sigma-rectangle list whose left-out pairs are proven unreachable in FP64, and
exactly the sub-list of the library's binning rule (lists and ranges bit
exact). Images: max abs error <= 2e-4 per channel. Gradients: relative L2 <= 1e-3 per tensor. Pixels where
the oracle sees a threshold within its ambiguity band are compared loosely
and counted (their upstream gradient is zero in the gradient checks).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_07021_gb300 import render, sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

from parity_util import (GpuView, check_decisions, check_grads, check_image, gpu_render,
                         gpu_view_lists, masked_dimg, pixel_mask_of_tiles, unpack_views)

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sgsplat.lib()
    oracle.lib()


def run_parity(scene, cams, seed=0, grads=True, tile_sels=None, storage="f32", ref_scene=None):
    """Forward (+ backward) on the GPU and in the oracle; returns reports."""
    ref_scene = scene if ref_scene is None else ref_scene
    ds, out = gpu_render(scene, cams, storage)
    results, _ = oracle.render(ref_scene, cams, tile_sel=tile_sels)
    gv = GpuView.plain(ds, cams, out)
    check_decisions(gv, cams, [(v, ref_scene, r) for v, r in enumerate(results)])
    imgs = unpack_views(out.img, cams, 3)
    Ts = unpack_views(out.T_final, cams, 1)
    lasts = unpack_views(out.last, cams, 1)
    rep = []
    for v, cam in enumerate(cams):
        mask = None if tile_sels is None else pixel_mask_of_tiles(cam, tile_sels[v])
        rep.append(check_image(imgs[v], Ts[v], lasts[v], results[v], cam, gpu_view_lists(gv, cams, v), mask))
    if not grads:
        return rep, None
    rng = np.random.default_rng(seed)
    dimgs = masked_dimg(rng, cams, results, tile_sels)
    _, g_orc = oracle.render(ref_scene, cams, dimgs=dimgs, tile_sel=tile_sels)
    same = all((c.width, c.height) == (cams[0].width, cams[0].height) for c in cams)
    if same:
        d = torch.from_numpy(np.stack(dimgs)).cuda()
    else:
        d = torch.from_numpy(np.concatenate([x.reshape(-1) for x in dimgs])).cuda()
    g_gpu = render.render_backward(ds, cams, out, d)
    torch.cuda.synchronize()
    grep = check_grads(g_gpu, g_orc)
    return rep, grep


def test_config0_forward():
    """1,000 Gaussians, 3 lobes each, 128x128, fx=fy=150 (forward only)."""
    scene, cams = synth.config0()
    rep, _ = run_parity(scene, cams, grads=False)
    assert rep[0]["max_abs_err"] <= 2e-4


def test_config0_forward_backward():
    scene, cams = synth.config0()
    run_parity(scene, cams, seed=1)


@pytest.mark.parametrize("seed", [0, 1])
def test_ragged_multi_batch_scene(seed):
    """Non-multiple-of-16 image, lists longer than one 256-entry batch, lobe mix
    0..4, soft masks, non-black background, early termination."""
    rng = np.random.default_rng(500 + seed)
    scene = synth.make_scene(rng, 6000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.4,
                             masks="uniform")
    cam = synth.make_camera(100, 70, 90.0, bg=(0.2, 0.4, 0.1))
    rep, grep = run_parity(scene, [cam], seed=seed)
    assert max(r["max_abs_err"] for r in rep) <= 2e-4


def test_multi_view_sums_gradients():
    rng = np.random.default_rng(42)
    scene = synth.make_scene(rng, 1500, lobes=synth.LOBE_MIX, means="cube", masks="uniform")
    cams = [synth.make_camera(64, 48, 60.0, viewmat=synth.look_at(eye, (0.0, 0.0, 4.0)))
            for eye in ((0.0, 0.0, 0.0), (1.0, 0.3, 0.5), (-0.8, -0.4, 0.2))]
    run_parity(scene, cams, seed=3)


def test_mixed_resolution_views():
    rng = np.random.default_rng(43)
    scene = synth.make_scene(rng, 800, lobes=2, means="cube", masks="uniform")
    cams = [synth.make_camera(64, 48, 60.0), synth.make_camera(33, 17, 30.0),
            synth.make_camera(16, 16, 20.0)]
    run_parity(scene, cams, seed=4)


def test_full_size_1080p_sampled():
    """500k Gaussians (32 clusters), 1920x1080, fx=1500: every tile list and
    range bit exact; image and gradients on a sample of tiles (the upstream
    gradient is zero elsewhere, so the oracle can compute them exactly)."""
    scene, cams, rng = synth.config1()
    cam = cams[0]
    sel = np.zeros(cam.n_tiles, bool)
    sel[np.random.default_rng(7).choice(cam.n_tiles, 48, replace=False)] = True
    sel[cam.n_tiles - 1] = True   # ragged bottom-right tile
    rep, grep = run_parity(scene, cams, seed=11, tile_sels=[sel])
    assert rep[0]["ambiguous"] <= 0.01 * rep[0]["pixels"]


# ---------------------------------------------------------------------------
# degenerate cases
# ---------------------------------------------------------------------------

def _empty_like(n_lobes=0):
    f = np.float32
    return synth.Scene(means=np.zeros((3, 0), f), scales=np.zeros((3, 0), f),
                       quats=np.zeros((4, 0), f), opac=np.zeros(0, f), gmask=np.zeros(0, f),
                       c0=np.zeros((3, 0), f), lobe_off=np.zeros(1, np.int32),
                       axis=np.zeros((3, 0), f), sharp=np.zeros(0, f), amp=np.zeros((3, 0), f),
                       lmask=np.zeros(0, f))


def test_empty_scene_renders_background():
    cam = synth.make_camera(40, 24, 50.0, bg=(0.1, 0.2, 0.3))
    ds, out = gpu_render(_empty_like(), [cam])
    img = out.img.cpu().numpy()[0]
    for ch, b in enumerate((0.1, 0.2, 0.3)):
        assert np.all(img[ch] == np.float32(b))
    assert torch.all(out.T_final == 1) and torch.all(out.last == 0)
    assert out.sizes["n_pairs"] == 0
    g = render.render_backward(ds, [cam], out, torch.ones_like(out.img))
    torch.cuda.synchronize()
    assert all(v.numel() == 0 for v in g.values())


def test_all_culled_and_zero_masks():
    rng = np.random.default_rng(5)
    scene = synth.make_scene(rng, 500, lobes=2, means="cube", cube_center=(0, 0, -4.0))
    cam = synth.make_camera(32, 32, 40.0)
    ds, out = gpu_render(scene, [cam])
    assert out.sizes["n_pairs"] == 0
    assert torch.all(out.T_final == 1)
    scene = synth.make_scene(rng, 500, lobes=2, means="cube")
    scene.gmask[:] = 0
    ds, out = gpu_render(scene, [cam])
    assert out.sizes["n_pairs"] == 0
    g = render.render_backward(ds, [cam], out, torch.ones_like(out.img))
    torch.cuda.synchronize()
    for k, v in g.items():
        assert torch.all(v == 0), k


def test_no_lobes_anywhere():
    rng = np.random.default_rng(6)
    scene = synth.make_scene(rng, 700, lobes=0, means="cube", masks="uniform")
    assert scene.n_lobes == 0
    run_parity(scene, [synth.make_camera(48, 40, 60.0)], seed=6)


def test_single_pixel_and_screen_covering_gaussian():
    rng = np.random.default_rng(8)
    scene = synth.make_scene(rng, 50, lobes=1, means="cube")
    scene.scales[:, 0] = 2.0      # one Gaussian larger than the image
    run_parity(scene, [synth.make_camera(1, 1, 2.0)], seed=8)
    run_parity(scene, [synth.make_camera(37, 29, 30.0)], seed=9)


@pytest.mark.parametrize("ppt", [(1, 1), (2, 2), (4, 4), (8, 8), (2, 8), (8, 1)])
def test_every_blend_shape(ppt):
    """Every pixels-per-thread variant of both blend kernels against the oracle."""
    rng = np.random.default_rng(600)
    scene = synth.make_scene(rng, 5000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.4,
                             masks="uniform")
    cam = synth.make_camera(70, 50, 70.0, bg=(0.3, 0.1, 0.2))
    old = sgsplat.sg_get_tuning()
    sgsplat.sg_set_tuning(*ppt)
    try:
        run_parity(scene, [cam], seed=12)
    finally:
        sgsplat.sg_set_tuning(**old)


@pytest.mark.parametrize("batches", [(32, 32), (128, 64), (64, 32)])
def test_every_batch_size(batches):
    """Every shared-memory batch size of both blend kernels against the oracle,
    in both the one-block-per-tile and the persistent forms."""
    rng = np.random.default_rng(610)
    scene = synth.make_scene(rng, 5000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.4,
                             masks="uniform")
    cam = synth.make_camera(70, 50, 70.0, bg=(0.3, 0.1, 0.2))
    old = sgsplat.sg_get_tuning()
    try:
        for persistent in (0, 1):
            sgsplat.sg_set_tuning(fwd_persistent=persistent, bwd_persistent=persistent, fwd_batch=batches[0],
                                  bwd_batch=batches[1])
            run_parity(scene, [cam], seed=14 + persistent)
    finally:
        sgsplat.sg_set_tuning(**old)


@pytest.mark.parametrize("storage", ["f16", "f16_bf16s"])
def test_half_precision_storage(storage):
    """Geometry and lobes stored in binary16 (sharpness optionally bfloat16),
    arithmetic in binary32: against the oracle fed the same rounded values."""
    rng = np.random.default_rng(650)
    scene = synth.make_scene(rng, 5000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.4,
                             masks="uniform")
    ref = synth.round_to_storage(scene, storage)
    cam = synth.make_camera(70, 50, 70.0, bg=(0.1, 0.1, 0.3))
    run_parity(scene, [cam], seed=13, storage=storage, ref_scene=ref)


def test_tuning_rejects_bad_shapes():
    with pytest.raises(sgsplat.SGError):
        sgsplat.sg_set_tuning(3, 4)
    with pytest.raises(sgsplat.SGError):
        sgsplat.sg_set_tuning(fwd_batch=48)
    with pytest.raises(sgsplat.SGError):
        sgsplat.sg_set_tuning(bwd_batch=128)
    sgsplat.sg_set_tuning()
    t = sgsplat.sg_get_tuning()
    assert (t["fwd_pixels_per_thread"], t["bwd_pixels_per_thread"], t["fwd_persistent"],
            t["bwd_persistent"]) == (4, 8, 1, 1)


def test_capacity_error_and_retry():
    scene, cams = synth.config0()
    ds = DeviceScene.from_host(scene)
    q = sgsplat.sg_workspace_query(ds, cams, 10)
    ws = torch.empty(q["ws_bytes"], dtype=torch.uint8, device="cuda")
    img = torch.empty(1, 3, 128, 128, device="cuda")
    T = torch.empty(1, 128, 128, device="cuda")
    last = torch.empty(1, 128, 128, dtype=torch.int32, device="cuda")
    st, out = sgsplat.sg_render_forward(ds, cams, ws, img, T, last, raise_on_error=False)
    assert st == sgsplat.SG_ERR_CAPACITY
    need = out["n_pairs"]
    assert need > 10
    ws = torch.empty(out["ws_bytes"], dtype=torch.uint8, device="cuda")
    st, out2 = sgsplat.sg_render_forward(ds, cams, ws, img, T, last, raise_on_error=False)
    assert st == sgsplat.SG_OK and out2["n_pairs"] == need
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    st, _ = sgsplat.sg_render_forward(ds, cams, small, img, T, last, raise_on_error=False)
    assert st == sgsplat.SG_ERR_WORKSPACE


def test_autograd_function_matches_direct_backward():
    scene, cams = synth.config0()
    ds = DeviceScene.from_host(scene)
    leaves = {k: getattr(ds, k).clone().requires_grad_(True) for k in DeviceScene.FLOAT_FIELDS}
    img, T, last = render.SGRasterize.apply(leaves["means"], leaves["scales"], leaves["quats"],
                                            leaves["opac"], leaves["gmask"], leaves["c0"],
                                            ds.lobe_off, leaves["axis"], leaves["sharp"],
                                            leaves["amp"], leaves["lmask"], cams)
    assert not T.requires_grad and not last.requires_grad
    target = torch.rand_like(img)
    loss = (img - target).abs().mean()
    loss.backward()
    d = torch.sign(img.detach() - target) / img.numel()
    out = render.render_forward(ds, cams)
    g = render.render_backward(ds, cams, out, d)
    torch.cuda.synchronize()
    for k in DeviceScene.FLOAT_FIELDS:
        a, b = leaves[k].grad, g[k]
        assert a is not None, k
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-7), k
    assert leaves["gmask"].grad.abs().sum() > 0 and leaves["lmask"].grad.abs().sum() > 0


def test_autograd_l1_loss_matches_oracle_adjoint():
    """A weighted L1 loss through SGRasterize (the autograd Function) against
    the FP64 oracle's adjoint of the same loss: every gradient, the
    soft-pruning masks m_g and m_l included (Sec. 3.3). Elements where the
    oracle sees a threshold within its ambiguity band, or where the image lies
    within 1e-3 of the target (the sign of the L1 derivative could differ),
    carry weight 0."""
    rng = np.random.default_rng(670)
    scene = synth.make_scene(rng, 3000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.4, masks="uniform")
    cam = synth.make_camera(72, 56, 70.0, bg=(0.1, 0.2, 0.3))
    res = oracle.render_forward(scene, cam, need_grad=True)
    target = rng.random((3, cam.height, cam.width))
    keep = ~res.ambiguous[None] & (np.abs(res.img - target) > 1e-3)
    w = keep / keep.sum()
    ds = DeviceScene.from_host(scene)
    leaves = {k: getattr(ds, k).clone().requires_grad_(True) for k in DeviceScene.FLOAT_FIELDS}
    img, T, last = render.SGRasterize.apply(leaves["means"], leaves["scales"], leaves["quats"],
                                            leaves["opac"], leaves["gmask"], leaves["c0"],
                                            ds.lobe_off, leaves["axis"], leaves["sharp"],
                                            leaves["amp"], leaves["lmask"], [cam])
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    wt = torch.from_numpy(w.astype(np.float32)).cuda()
    loss = ((img[0] - tgt).abs() * wt).sum()
    loss.backward()
    torch.cuda.synchronize()
    got_img = img[0].detach().cpu().numpy()
    assert np.array_equal(np.sign(got_img - target)[keep], np.sign(res.img - target)[keep])
    g_orc = oracle.render_backward(res, scene, cam, np.sign(res.img - target) * w)
    rep = check_grads({k: leaves[k].grad for k in DeviceScene.FLOAT_FIELDS}, g_orc)
    assert set(rep) >= {"gmask", "lmask"}
    assert np.abs(g_orc["gmask"]).sum() > 0 and np.abs(g_orc["lmask"]).sum() > 0


# ---------------------------------------------------------------------------
# importance score (App. A.2), fused into the forward blend
# ---------------------------------------------------------------------------

def unambiguous_gaussians(results, n):
    """Gaussians that reach no ambiguous pixel of any view: where every pixel a
    Gaussian can blend at (alpha >= 1/255 in FP64, with a margin) has only
    unambiguous decisions, its sum of weights has one correct value."""
    ok = np.ones(n, bool)
    for r in results:
        H, W = r.ambiguous.shape
        tiles_x = (W + 15) // 16
        for py, px in zip(*np.nonzero(r.ambiguous)):
            t = (py // 16) * tiles_x + px // 16
            ids = r.ids[r.ranges[t, 0]:r.ranges[t, 1]]
            dx, dy = px - r.xy[ids, 0], py - r.xy[ids, 1]
            con = r.conic[ids]
            q = con[:, 0] * dx * dx + 2 * con[:, 1] * dx * dy + con[:, 2] * dy * dy
            with np.errstate(all="ignore"):
                bound = 2.0 * np.log(255.0 * r.op[ids]) * 1.01 + 0.1
            ok[ids[~(q > bound)]] = False
    return ok


def check_importance(got, expect, ok):
    """Element-wise where the value is unique, and in L2 over all Gaussians."""
    assert np.isfinite(got).all()
    assert ok.mean() > 0.5
    np.testing.assert_allclose(got[ok], expect[ok], rtol=1e-4, atol=1e-6 * max(expect.max(), 1.0))
    assert np.linalg.norm(got - expect) <= 1e-3 * np.linalg.norm(expect)
    assert (got[expect == 0] == 0).all()

@pytest.mark.parametrize("fwd_ppt", [1, 2, 4])
def test_importance_matches_oracle(fwd_ppt):
    rng = np.random.default_rng(660)
    scene = synth.make_scene(rng, 4000, lobes=synth.LOBE_MIX, means="cube", cube_side=1.4,
                             masks="uniform")
    cams = [synth.make_camera(72, 56, 70.0),
            synth.make_camera(50, 40, 60.0, viewmat=synth.look_at((0.3, -0.2, 0.2), (0, 0, 4.0)))]
    ds = DeviceScene.from_host(scene)
    imp = torch.full((scene.n,), float("nan"), device="cuda")
    old = sgsplat.sg_get_tuning()
    sgsplat.sg_set_tuning(fwd_pixels_per_thread=fwd_ppt)
    try:
        out = render.render_forward(ds, cams, importance=imp)
        ref = render.render_forward(ds, cams)
        torch.cuda.synchronize()
    finally:
        sgsplat.sg_set_tuning(**old)
    # the importance variant renders the same image
    assert torch.equal(out.img, ref.img) and torch.equal(out.last, ref.last)
    results, _ = oracle.render(scene, cams)
    expect = sum(r.importance for r in results)
    got = imp.cpu().numpy().astype(np.float64)
    check_importance(got, expect, unambiguous_gaussians(results, scene.n))
