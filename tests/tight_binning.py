"""The library's tight tile binning, restated in numpy binary32 for the tests.

This is NOT part of the oracle. The oracle's tile lists follow the rasterizer
the paper keeps (Sec. 3.1, Sec. 4: 3DGS gives a Gaussian a pair in every tile
of its 3-sigma rectangle). The library bins more tightly: of the rectangle's
tiles it keeps only those whose box of pixel centres meets the ellipse
q = d^T conic d <= 2 ln(255 o'), outside which alpha < 1/255 at every pixel (so
the blend would skip the pair at every pixel of the tile). The ellipse is
enlarged (q bound x 1.01 + 0.01, 0.02 px) so binary32 rounding can only keep
extra tiles.

The parity tests use this module to state which ordered sub-list of the
oracle's lists the library must produce, bit for bit; the oracle alone proves,
in FP64, that every pair the sub-list leaves out is unreachable
(parity_util.check_decisions). Every step below is one binary32
round-to-nearest operation in the library's order, so the kept tiles agree
exactly.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def _hexf(h):
    return F32(float.fromhex(h))


# exact binary32 constants of the binning recipe
C7, C5, C3 = _hexf("0x1.24924ap-3"), _hexf("0x1.99999ap-3"), _hexf("0x1.555556p-2")   # 1/7, 1/5, 1/3
INV_LN2, LN2X2 = _hexf("0x1.715476p+0"), _hexf("0x1.62e430p+0")                         # 1/ln 2, 2 ln 2
GROW, ADD, PAD = _hexf("0x1.028f5cp+0"), _hexf("0x1.47ae14p-7"), _hexf("0x1.47ae14p-6")  # 1.01, 0.01, 0.02
INV16 = _hexf("0x1p-4")


def log2_recipe(x):
    """log2 of positive normal binary32 x: exponent + ln(m)/ln 2 for the
    mantissa m in [1, 2), ln m = 2 atanh(s), s = (m - 1)/(m + 1), series to s^7."""
    x = np.asarray(x, F32)
    u = x.view(np.uint32)
    e = (((u >> np.uint32(23)) & np.uint32(255)).astype(np.int32) - 127).astype(F32)
    m = ((u & np.uint32(0x007FFFFF)) | np.uint32(0x3F800000)).view(F32)
    one = F32(1.0)
    s_ = (m - one) / (m + one)
    s2 = s_ * s_
    P = s2 * C7 + C5
    P = P * s2 + C3
    P = P * s2 + one
    lnm = (F32(2.0) * s_) * P
    return e + lnm * INV_LN2


def reach_threshold(opd):
    """Enlarged bound on q, 2 ln(255 o') x 1.01 + 0.01 (binary32); -1 where
    o' < 1/255 (the pair reaches no pixel)."""
    opd = np.asarray(opd, F32)
    with np.errstate(all="ignore"):
        t0 = LN2X2 * log2_recipe(F32(255.0) * opd)
        t = t0 * GROW + ADD
    return np.where(opd >= F32(1.0 / 255.0), t, F32(-1.0)).astype(F32)


def reach_rows(dec, reach_t):
    """For every tile row of every visible Gaussian's rectangle (in Gaussian,
    then row order), the columns [c0, c1) the enlarged ellipse reaches.
    Returns (gaussian id, ty, c0, c1)."""
    f = F32
    ids_v = np.nonzero(dec.visible)[0]
    r = dec.rect[ids_v].astype(np.int64)
    h = r[:, 3] - r[:, 1]
    g = np.repeat(ids_v, h)
    start = np.repeat(np.cumsum(h) - h, h)
    ty = np.repeat(r[:, 1], h) + (np.arange(int(h.sum()), dtype=np.int64) - start)
    x0 = dec.rect[g, 0].astype(np.int64)
    x1 = dec.rect[g, 2].astype(np.int64)
    with np.errstate(all="ignore"):
        A, B, C = (dec.conic32[g, k].astype(f) for k in range(3))
        x, y = dec.xy32[g, 0].astype(f), dec.xy32[g, 1].astype(f)
        t = reach_t[g].astype(f)
        det = A * C - B * B
        ok = (A > 0) & (C > 0) & (det > 0) & np.isfinite(t) & np.isfinite(det)
        At = A * t
        ymax = np.sqrt(At / det)
        xmax = np.sqrt((C * t) / det)
        m = (B * xmax) / C
        iA = f(1.0) / A
        mode = np.where(~(t >= 0), 0, np.where(ok & np.isfinite(ymax) & np.isfinite(m) & np.isfinite(At)
                                                & np.isfinite(iA), 1, 2))
        lo = np.maximum((f(16.0) * ty.astype(f) - y) - PAD, -ymax)
        hi = np.minimum(((f(16.0) * ty.astype(f) + f(15.0)) - y) + PAD, ymax)
        nonempty = lo <= hi
        dr = np.minimum(np.maximum(-m, lo), hi)
        dl = np.minimum(np.maximum(m, lo), hi)
        sr = np.sqrt(np.maximum(f(0.0), At - det * (dr * dr)))
        sl = np.sqrt(np.maximum(f(0.0), At - det * (dl * dl)))
        xr = (x + (sr - B * dr) * iA) + PAD
        xl = (x - (sl + B * dl) * iA) - PAD
        fx0 = (16 * x0 - 16).astype(f)
        fx1 = (16 * x1).astype(f)
        a = np.ceil((np.minimum(np.maximum(xl, fx0), fx1) - f(15.0)) * INV16)
        b = np.floor(np.minimum(np.maximum(xr, fx0), fx1) * INV16)
    a = np.where(mode == 1, a, 0).astype(np.int64)
    b = np.where(mode == 1, b, 0).astype(np.int64)
    c0 = np.maximum(x0, a)
    c1 = np.maximum(c0, np.minimum(x1, b + 1))
    c0 = np.where(mode == 2, x0, np.where((mode == 1) & nonempty, c0, x0))
    c1 = np.where(mode == 2, x1, np.where((mode == 1) & nonempty, c1, x0))
    return g, ty, c0, c1


def binning_bound(scene):
    """The per-Gaussian bound the library stores in its record (from o' = m_g o)."""
    opd = scene.gmask.astype(F32) * scene.opac.astype(F32)
    return reach_threshold(opd)


def kept_pairs(dec, reach_t, cam, keys, ids):
    """Boolean mask over the oracle's sorted full-rectangle pairs (keys, ids):
    True where the library's tight binning keeps the pair."""
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    if len(tiles) == 0:
        return np.zeros(0, bool)
    _, _, c0, c1 = reach_rows(dec, reach_t)
    h = np.where(dec.visible, dec.rect[:, 3] - dec.rect[:, 1], 0).astype(np.int64)
    row_start = np.cumsum(h) - h
    tx, ty = tiles % cam.tiles_x, tiles // cam.tiles_x
    row = row_start[ids] + (ty - dec.rect[ids, 1])
    return (c0[row] <= tx) & (tx < c1[row])


def touched(dec, reach_t):
    """Tiles each Gaussian gets under the tight binning ([N] int64)."""
    g, _, c0, c1 = reach_rows(dec, reach_t)
    return np.bincount(g, weights=(c1 - c0), minlength=len(dec.visible)).astype(np.int64)
