"""Helpers for the GPU-vs-oracle parity tests: run the CUDA path through the C
ABI, read its workspace, and compare with the FP64 oracle."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2509_07021_gb300 import render, sgsplat
from paper_2509_07021_gb300.sgsplat import DeviceScene

IMG_TOL = 2e-4      # max abs per channel (images)
GRAD_TOL = 1e-3     # relative L2 per gradient tensor


def u32(t: torch.Tensor) -> np.ndarray:
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


class GpuView:
    """Per-view slices of a finished forward's workspace."""

    def __init__(self, ds: DeviceScene, cams, out: render.ForwardOut):
        ws = out.ws
        lay = sgsplat.sg_workspace_layout(ds, cams, ws.numel())
        M, K, T = out.sizes["n_entries"], out.sizes["n_pairs"], out.sizes["n_tiles"]
        torch.cuda.synchronize()
        self.rec = ws[lay["rec"]:lay["rec"] + 48 * M].view(torch.float32).reshape(M, 12).cpu().numpy()
        self.tt = u32(ws[lay["tiles_touched"]:lay["tiles_touched"] + 4 * M])
        rect = u32(ws[lay["rect"]:lay["rect"] + 8 * M]).reshape(M, 2)
        self.rect = np.stack([rect[:, 0] & 0xFFFF, rect[:, 1] & 0xFFFF, rect[:, 0] >> 16,
                              rect[:, 1] >> 16], 1).astype(np.int64)
        self.ranges = u32(ws[lay["ranges"]:lay["ranges"] + 8 * T]).reshape(T, 2).astype(np.int64)
        self.pair_tile = u32(ws[lay["pair_tile"]:lay["pair_tile"] + 4 * K]).astype(np.int64)
        self.pair_entry = u32(ws[lay["pair_entry"]:lay["pair_entry"] + 4 * K]).astype(np.int64)
        self.n = ds.n
        self.cams = cams
        self.K = K


def tile_offsets(cams):
    offs = [0]
    for c in cams:
        offs.append(offs[-1] + c.n_tiles)
    return offs


def _box_min_q(con, xy, tx, ty):
    """FP64 minimum of q = A dx^2 + 2 B dx dy + C dy^2 over the box of pixel
    centres of tile (tx, ty), dx = x - x_g, dy = y - y_g (vectorised)."""
    A, B, C = con[:, 0], con[:, 1], con[:, 2]
    lx, hx = tx * 16.0 - xy[:, 0], tx * 16.0 + 15.0 - xy[:, 0]
    ly, hy = ty * 16.0 - xy[:, 1], ty * 16.0 + 15.0 - xy[:, 1]
    best = np.where((lx <= 0) & (hx >= 0) & (ly <= 0) & (hy >= 0), 0.0, np.inf)
    for fx in (lx, hx):
        dy = np.clip(-B * fx / C, ly, hy)
        best = np.minimum(best, A * fx * fx + 2 * B * fx * dy + C * dy * dy)
    for fy in (ly, hy):
        dx = np.clip(-B * fy / A, lx, hx)
        best = np.minimum(best, A * dx * dx + 2 * B * dx * fy + C * fy * fy)
    return best


def gpu_view_lists(gv: GpuView, cams, v):
    """(ranges [n_tiles, 2], ids [pairs]) of view v from the GPU workspace, ids
    relative to the view (Gaussian index)."""
    toffs = tile_offsets(cams)
    rg = gv.ranges[toffs[v]:toffs[v + 1]]
    return rg, gv.pair_entry - v * gv.n


def check_decisions(gv: GpuView, scene, cams, results):
    """Cull, radius, rectangle, depth key, binary32 centre/conic/opacity: bit exact.

    Tile lists: the oracle keeps every tile of the 3-sigma rectangle; the GPU
    keeps only tiles whose pixel-centre box its enlarged alpha >= 1/255 ellipse
    meets. So each GPU list must be an order-preserving sub-list of the oracle's
    list for that tile, every pair it leaves out must be one that the FP64
    geometry proves can blend at no pixel of the tile (the minimum of q over the
    tile's pixel-centre box exceeds 2 ln(255 o')), and tiles_touched must count
    the GPU pairs of each entry."""
    toffs = tile_offsets(cams)
    total_orc = 0
    for v, (cam, res) in enumerate(zip(cams, results)):
        sl = slice(v * gv.n, (v + 1) * gv.n)
        dec = res.dec
        rect = gv.rect[sl]
        vis = (rect[:, 2] > rect[:, 0]) & (rect[:, 3] > rect[:, 1])
        np.testing.assert_array_equal(vis, dec.visible, err_msg=f"view {v}: visibility")
        rec = gv.rec[sl][vis]
        np.testing.assert_array_equal(rect[vis], dec.rect[vis], err_msg=f"view {v}: rect")
        np.testing.assert_array_equal(rec[:, 9].astype(np.int64), dec.radius[vis], err_msg="radius")
        np.testing.assert_array_equal(rec[:, 10].view(np.uint32), dec.depth_bits[vis], err_msg="depth")
        np.testing.assert_array_equal(rec[:, 0:2].view(np.uint32),
                                      dec.xy32[vis].astype(np.float32).view(np.uint32), err_msg="xy")
        np.testing.assert_array_equal(rec[:, [2, 3, 4]].view(np.uint32),
                                      dec.conic32[vis].astype(np.float32).view(np.uint32), err_msg="conic")
        opd = (scene.gmask.astype(np.float32) * scene.opac.astype(np.float32))[vis]
        np.testing.assert_array_equal(rec[:, 5], opd)
        area = (dec.rect[:, 2] - dec.rect[:, 0]) * (dec.rect[:, 3] - dec.rect[:, 1])
        tt = gv.tt[sl]
        assert np.all(tt[~vis] == 0) and np.all(tt[vis] <= area[vis])
        # GPU lists of this view
        rg, ids_all = gpu_view_lists(gv, cams, v)
        lens = rg[:, 1] - rg[:, 0]
        nonempty = lens > 0
        idx = np.concatenate([np.arange(s, s + l) for s, l in zip(rg[nonempty, 0], lens[nonempty])]) \
            if nonempty.any() else np.zeros(0, np.int64)
        g_ids = ids_all[idx]
        g_tile = gv.pair_tile[idx] - toffs[v]
        np.testing.assert_array_equal(g_tile, np.repeat(np.nonzero(nonempty)[0], lens[nonempty]))
        np.testing.assert_array_equal(np.bincount(g_ids, minlength=gv.n), tt, err_msg="tiles_touched")
        # oracle lists: (tile, id) -> position
        o_tile = (res.keys >> np.uint64(32)).astype(np.int64)
        o_ids = res.ids.astype(np.int64)
        total_orc += len(o_ids)
        N = gv.n
        o_key = o_tile * N + o_ids
        order = np.argsort(o_key, kind="stable")
        g_key = g_tile * N + g_ids
        at = np.searchsorted(o_key[order], g_key)
        assert np.all(at < len(o_key)) and np.all(o_key[order][np.minimum(at, len(o_key) - 1)] == g_key), \
            "a GPU pair is not in the oracle's lists"
        pos = order[at]
        same = np.diff(g_tile) == 0
        assert np.all(np.diff(pos)[same] > 0), "GPU list order differs from the oracle's"
        # every left-out pair blends nowhere in its tile (FP64 geometry)
        kept = np.zeros(len(o_ids), bool)
        kept[pos] = True
        drop = ~kept
        if drop.any():
            gid, t = o_ids[drop], o_tile[drop]
            qmin = _box_min_q(res.conic[gid], res.xy[gid], t % cam.tiles_x, t // cam.tiles_x)
            op = res.op[gid]
            thr = np.where(op > 1.0 / 255.0, 2.0 * np.log(np.maximum(255.0 * op, 1e-300)), -1.0)
            bad = ~(qmin > thr)
            assert not bad.any(), f"view {v}: {int(bad.sum())} left-out pairs could blend"
    # pairs of all views are contiguous and ordered by global tile
    assert gv.K <= total_orc
    assert np.all(np.diff(gv.pair_tile) >= 0)


def last_ids(last, ranges, ids, cam):
    """Gaussian blended last at each pixel (-1: none) from per-pixel list
    positions `last` and that renderer's tile lists."""
    H, W = last.shape
    ty, tx = np.meshgrid(np.arange(H) // 16, np.arange(W) // 16, indexing="ij")
    tile = ty * cam.tiles_x + tx
    out = np.full((H, W), -1, np.int64)
    m = last > 0
    out[m] = ids[ranges[tile[m], 0] + last[m] - 1]
    return out


def pixel_mask_of_tiles(cam, tile_sel):
    m = np.repeat(np.repeat(tile_sel.reshape(cam.tiles_y, cam.tiles_x), 16, 0), 16, 1)
    return m[:cam.height, :cam.width].astype(bool)


def check_image(img, T, last, res, cam, mask=None, tol=IMG_TOL, gpu_lists=None):
    """img [3,H,W], T [H,W], last [H,W] from the GPU against one oracle view.
    Unambiguous pixels: image within tol, T within tol, and the last blended
    Gaussian the same (through both renderers' tile lists when the GPU's are
    given, `gpu_lists` = (ranges, ids) of the view; else whether any was).
    Ambiguous pixels (a threshold within the oracle's band): counted, and the
    image must stay within one blended contribution (0.02) of the oracle."""
    amb = res.ambiguous
    sel = np.ones(amb.shape, bool) if mask is None else mask
    ok = sel & ~amb
    err = np.abs(img - res.img)
    assert ok.sum() > 0
    max_err = err[:, ok].max()
    assert max_err <= tol, f"image max abs error {max_err:.3e} > {tol}"
    if gpu_lists is not None:
        g = last_ids(last.astype(np.int64), gpu_lists[0], gpu_lists[1], cam)
        o = last_ids(res.last, res.ranges.astype(np.int64), res.ids.astype(np.int64), cam)
        np.testing.assert_array_equal(g[ok], o[ok])
    else:
        np.testing.assert_array_equal(last[ok] > 0, res.last[ok] > 0)
    assert np.abs(T - res.T_final)[ok].max() <= tol
    n_amb = int((sel & amb).sum())
    if n_amb:
        assert err[:, sel & amb].max() <= 0.02
    assert n_amb <= max(2, 0.01 * sel.sum()), f"{n_amb} ambiguous pixels"
    return {"max_abs_err": float(max_err), "mean_abs_err": float(err[:, ok].mean()),
            "ambiguous": n_amb, "pixels": int(sel.sum())}


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def check_grads(g_gpu: dict, g_orc: dict, tol=GRAD_TOL, skip=()):
    report = {}
    for k, ref in g_orc.items():
        if k in skip:
            continue
        got = g_gpu[k].detach().cpu().numpy().astype(np.float64)
        assert got.shape == ref.shape, k
        if ref.size == 0:
            report[k] = 0.0
            continue
        if np.linalg.norm(ref) == 0:
            assert np.abs(got).max() <= 1e-6, (k, np.abs(got).max())
            report[k] = 0.0
            continue
        r = rel_l2(got, ref)
        report[k] = r
        assert r <= tol, f"{k}: relative L2 {r:.3e} > {tol}"
    return report


def gpu_render(scene, cams, storage="f32"):
    ds = DeviceScene.from_host(scene, storage=storage)
    out = render.render_forward(ds, cams)
    torch.cuda.synchronize()
    return ds, out


def unpack_views(t, cams, ch):
    """Flat or [V,...] output -> list of per-view numpy arrays ([3,H,W] or [H,W])."""
    a = t.detach().cpu().numpy()
    if a.ndim > 1:
        return [a[v] for v in range(len(cams))]
    out, o = [], 0
    for c in cams:
        n = c.width * c.height * ch
        x = a[o:o + n]
        out.append(x.reshape(3, c.height, c.width) if ch == 3 else x.reshape(c.height, c.width))
        o += n
    return out


def masked_dimg(rng, cams, results, tile_sels=None, std=0.01):
    """Upstream gradients N(0, std), zero at the oracle's ambiguous pixels (and
    outside the selected tiles when given)."""
    out = []
    for i, (cam, res) in enumerate(zip(cams, results)):
        d = rng.normal(0.0, std, (3, cam.height, cam.width)).astype(np.float32)
        keep = ~res.ambiguous
        if tile_sels is not None:
            keep &= pixel_mask_of_tiles(cam, tile_sels[i])
        d *= keep[None]
        out.append(d)
    return out
