"""Helpers for the GPU-vs-oracle parity tests: run the CUDA path through the C
ABI, read its workspace, and compare with the FP64 oracle."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import tight_binning
from paper_2509_07021_gb300 import render, sgsplat
from paper_2509_07021_gb300.sgsplat import NO_OFFSET, DeviceScene

IMG_TOL = 2e-4      # max abs per channel (images)
GRAD_TOL = 1e-3     # relative L2 per gradient tensor


def u32(t: torch.Tensor) -> np.ndarray:
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


class GpuView:
    """Slices of a finished forward's workspace: every entry's record,
    tiles_touched and rectangle, the tile ranges and the sorted pairs.
    Entries are numbered view after view (view_n[v] Gaussians each)."""

    def __init__(self, ws, lay, M, K, T, view_n):
        torch.cuda.synchronize()
        self.rec = ws[lay["rec"]:lay["rec"] + 48 * M].view(torch.float32).reshape(M, 12).cpu().numpy()
        self.tt = u32(ws[lay["tiles_touched"]:lay["tiles_touched"] + 4 * M])
        rect = u32(ws[lay["rect"]:lay["rect"] + 8 * M]).reshape(M, 2)
        self.rect = np.stack([rect[:, 0] & 0xFFFF, rect[:, 1] & 0xFFFF, rect[:, 0] >> 16,
                              rect[:, 1] >> 16], 1).astype(np.int64)
        self.ranges = u32(ws[lay["ranges"]:lay["ranges"] + 8 * T]).reshape(T, 2).astype(np.int64)
        if lay["pair_tile"] == NO_OFFSET:
            # sorted by counting: no tile ids are kept, pair k's tile is the
            # tile whose range holds k (-1 where no range does)
            self.pair_tile = np.full(K, -1, np.int64)
            for t in np.nonzero(self.ranges[:, 1] > self.ranges[:, 0])[0]:
                self.pair_tile[self.ranges[t, 0]:self.ranges[t, 1]] = t
        else:
            self.pair_tile = u32(ws[lay["pair_tile"]:lay["pair_tile"] + 4 * K]).astype(np.int64)
        self.pair_entry = u32(ws[lay["pair_entry"]:lay["pair_entry"] + 4 * K]).astype(np.int64)
        self.view_n = [int(n) for n in view_n]
        self.ent_off = np.concatenate([[0], np.cumsum(self.view_n)]).astype(np.int64)
        self.K = K

    @classmethod
    def plain(cls, ds: DeviceScene, cams, out: render.ForwardOut):
        lay = sgsplat.sg_workspace_layout(ds, cams, out.ws.numel())
        return cls(out.ws, lay, out.sizes["n_entries"], out.sizes["n_pairs"], out.sizes["n_tiles"],
                   [ds.n] * len(cams))

    @classmethod
    def batched(cls, br: render.BatchedRenderer):
        lay = sgsplat.sg_batched_workspace_layout(br.scenes, br.cams, br.view_scene, br.ws.numel())
        K, st = br.status()
        assert st == sgsplat.SG_OK
        view_n = [br.scenes[s].n for s in br.view_scene]
        return cls(br.ws, lay, sum(view_n), K, sum(c.n_tiles for c in br.cams), view_n)


def tile_offsets(cams):
    offs = [0]
    for c in cams:
        offs.append(offs[-1] + c.n_tiles)
    return offs


def gpu_view_lists(gv: GpuView, cams, v):
    """(ranges [n_tiles, 2], ids [pairs]) of view v from the GPU workspace, ids
    relative to the view (Gaussian index)."""
    toffs = tile_offsets(cams)
    rg = gv.ranges[toffs[v]:toffs[v + 1]]
    return rg, gv.pair_entry - gv.ent_off[v]


def box_min_q(con, xy, tx, ty):
    """FP64 minimum of q = A dx^2 + 2 B dx dy + C dy^2 over the box of pixel
    centres of tile (tx, ty) (positive-definite conic)."""
    A, B, C = con[:, 0], con[:, 1], con[:, 2]
    lx, hx = tx * 16.0 - xy[:, 0], tx * 16.0 + 15.0 - xy[:, 0]
    ly, hy = ty * 16.0 - xy[:, 1], ty * 16.0 + 15.0 - xy[:, 1]
    best = np.where((lx <= 0) & (hx >= 0) & (ly <= 0) & (hy >= 0), 0.0, np.inf)
    with np.errstate(all="ignore"):
        for fx in (lx, hx):
            dy = np.clip(-B * fx / C, ly, hy)
            best = np.minimum(best, A * fx * fx + 2 * B * fx * dy + C * dy * dy)
        for fy in (ly, hy):
            dx = np.clip(-B * fy / A, lx, hx)
            best = np.minimum(best, A * dx * dx + 2 * B * dx * fy + C * fy * fy)
    return best


def unreachable(res, cam, tiles, ids):
    """FP64 proof that pair (tile, Gaussian) blends at no pixel of the tile:
    its conic is positive definite and q > 2 ln(255 o') on the whole box of
    pixel centres, so alpha = o' exp(-q/2) < 1/255 everywhere (the skip rule)."""
    con, xy, op = res.conic[ids], res.xy[ids], res.op[ids]
    pd = (con[:, 0] > 0) & (con[:, 2] > 0) & (con[:, 0] * con[:, 2] - con[:, 1] ** 2 > 0)
    with np.errstate(all="ignore"):
        thr = 2.0 * np.log(255.0 * op)
    q = box_min_q(con, xy, tiles % cam.tiles_x, tiles // cam.tiles_x)
    return pd & (q > thr)


def check_decisions(gv: GpuView, cams, checks):
    """checks: (view index, scene, oracle ViewResult) of the views to compare.
    Against the oracle: cull, radius, rectangle, depth key, binary32
    centre/conic/opacity bit exact; every GPU tile list an ordered sub-list of
    the oracle's full 3-sigma-rectangle list, every pair it leaves out proven
    unreachable in FP64; and, against the library's own binning rule restated
    in tight_binning, the kept pairs, tiles_touched and ranges bit exact."""
    toffs = tile_offsets(cams)
    for v, scene, res in checks:
        cam = cams[v]
        n = gv.view_n[v]
        bound = tight_binning.binning_bound(scene)
        sl = slice(gv.ent_off[v], gv.ent_off[v] + n)
        dec = res.dec
        rect = gv.rect[sl]
        vis = (rect[:, 2] > rect[:, 0]) & (rect[:, 3] > rect[:, 1])
        np.testing.assert_array_equal(vis, dec.visible, err_msg=f"view {v}: visibility")
        rec = gv.rec[sl][vis]
        np.testing.assert_array_equal(rect[vis], dec.rect[vis], err_msg=f"view {v}: rect")
        np.testing.assert_array_equal(rec[:, 10].astype(np.int64), dec.radius[vis], err_msg="radius")
        np.testing.assert_array_equal(rec[:, 11].view(np.uint32), dec.depth_bits[vis], err_msg="depth")
        np.testing.assert_array_equal(rec[:, 0:2].view(np.uint32),
                                      dec.xy32[vis].astype(np.float32).view(np.uint32), err_msg="xy")
        np.testing.assert_array_equal(rec[:, [2, 3, 4]].view(np.uint32),
                                      dec.conic32[vis].astype(np.float32).view(np.uint32), err_msg="conic")
        opd = (scene.gmask.astype(np.float32) * scene.opac.astype(np.float32))[vis]
        np.testing.assert_array_equal(rec[:, 6], opd)
        np.testing.assert_array_equal(rec[:, 5].view(np.uint32), bound[vis].view(np.uint32),
                                      err_msg="tile-binning bound")
        # the GPU's pairs of this view, in order
        rg = gv.ranges[toffs[v]:toffs[v + 1]]
        lens = rg[:, 1] - rg[:, 0]
        nonempty = lens > 0
        idx = np.concatenate([np.arange(s, s + l) for s, l in zip(rg[nonempty, 0], lens[nonempty])]) \
            if nonempty.any() else np.zeros(0, np.int64)
        g_ids = gv.pair_entry[idx] - gv.ent_off[v]
        g_tiles = gv.pair_tile[idx] - toffs[v]
        np.testing.assert_array_equal(g_tiles, np.repeat(np.arange(cam.n_tiles), lens), err_msg="pair tiles")
        # (1) an ordered sub-list of the oracle's lists (the paper's rule)
        o_tiles = (res.keys >> np.uint64(32)).astype(np.int64)
        o_code = o_tiles * n + res.ids
        g_code = g_tiles * n + g_ids
        srt = np.argsort(o_code, kind="stable")
        at = np.searchsorted(o_code[srt], g_code)
        at = np.minimum(at, max(len(o_code) - 1, 0))
        assert len(g_code) == 0 or np.array_equal(o_code[srt][at], g_code), f"view {v}: a GPU pair the oracle lacks"
        pos = srt[at] if len(g_code) else np.zeros(0, np.int64)
        assert np.all(np.diff(pos) > 0), f"view {v}: GPU lists out of the oracle's order"
        # (2) every pair left out blends at no pixel of its tile (FP64)
        left = np.ones(len(o_code), bool)
        left[pos] = False
        proven = unreachable(res, cam, o_tiles[left], res.ids[left])
        assert proven.all(), f"view {v}: {int((~proven).sum())} left-out pairs not proven unreachable"
        # (3) exactly the library's binning rule
        keep = tight_binning.kept_pairs(dec, bound, cam, res.keys, res.ids)
        np.testing.assert_array_equal(~left, keep, err_msg=f"view {v}: kept pairs")
        np.testing.assert_array_equal(gv.tt[sl], tight_binning.touched(dec, bound),
                                      err_msg=f"view {v}: tiles_touched")
        np.testing.assert_array_equal(gv.tt[sl], np.bincount(g_ids, minlength=n))
        assert np.all(gv.tt[sl] <= dec.touched)
    # pairs of all views are contiguous and ordered by global tile
    assert gv.K == int((gv.ranges[:, 1] - gv.ranges[:, 0]).sum())
    assert np.all(np.diff(gv.pair_tile[:gv.K]) >= 0)
    # every range starts where the tiles before it end; a tile with no pair holds (0, 0)
    lens = gv.ranges[:, 1] - gv.ranges[:, 0]
    ne = lens > 0
    np.testing.assert_array_equal(gv.ranges[ne, 0], (np.cumsum(lens) - lens)[ne], err_msg="range starts")
    np.testing.assert_array_equal(gv.ranges[~ne], 0, err_msg="tiles with no pair")


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


def check_image(img, T, last, res, cam, gpu_lists, mask=None, tol=IMG_TOL):
    """img [3,H,W], T [H,W], last [H,W] from the GPU against one oracle view.
    gpu_lists = (ranges, ids) of the view's GPU tile lists: `last` counts
    positions in each renderer's own lists, so the pixel's last blended
    Gaussian is compared by identity.
    Unambiguous pixels: image and T within tol, the same last blended Gaussian.
    Ambiguous pixels (a threshold within the oracle's band): counted, and the
    image must stay within one blended contribution (0.02) of the oracle."""
    amb = res.ambiguous
    sel = np.ones(amb.shape, bool) if mask is None else mask
    ok = sel & ~amb
    err = np.abs(img - res.img)
    assert ok.sum() > 0
    max_err = err[:, ok].max()
    assert max_err <= tol, f"image max abs error {max_err:.3e} > {tol}"
    g = last_ids(last.astype(np.int64), gpu_lists[0], gpu_lists[1], cam)
    o = last_ids(res.last, res.ranges.astype(np.int64), res.ids.astype(np.int64), cam)
    np.testing.assert_array_equal(g[ok], o[ok])
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
