"""Plain, slow CPU oracle of the SG-splatting rasterizer (FP64).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
baseline use it; the library path never imports it and has no fallback to it.
It shares no code with the CUDA path (the only common module is the seeded
input generator, which holds none of the method's arithmetic).

What it follows:
  * SG lobe and colour model, Eq. 1-2 (Sec. 3.2): c(v) = c0 + sum_i a_i e^{s_i(mu_i.v - 1)}.
    The degree-3 SH colour of the 3DGS baseline it replaces is in sg_sh_oracle.py.
    Soft-pruning masks (a differentiable form of Sec. 3.3's pruning): m_l multiplies the
    whole lobe term, m_g multiplies opacity.
  * Primitive model and front-to-back compositing, Sec. 3.1: a Gaussian with centre mu,
    covariance Sigma = R S S^T R^T, opacity o, projected with the EWA Jacobian and blended
    as C = sum_i c_i alpha_i prod_{j<i}(1 - alpha_j).
  * The compositing rules inherited from 3DGS that the paper keeps (0.3 px low-pass
    dilation, 3-sigma radius, 16x16 tiles, 1/255 skip, 0.99 clamp, 1e-4 stop, near plane
    0.2, 1.3x guard band): the paper states only the blend sum, so these are read as the
    rules of the rasterizer it builds on.

Discrete decisions (cull, radius, tile rectangle, depth key) are taken with the
binary32 recipe below, the same recipe the GPU uses, so that they can be
compared bit for bit; every value that feeds an image or a gradient is FP64.
Tile lists follow the rasterizer the paper keeps: a visible Gaussian gets a
pair in every tile of its 3-sigma rectangle, each tile's list in ascending
(depth, index) order.

The adjoint: per-Gaussian formulas (projection, conic, SG colour) are written
once in torch float64 and differentiated by autograd; the per-pixel blend
adjoint is written out in sg_blend_oracle.c. Both are pinned by FP64 central
finite differences in the tests.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from .sg_sh_oracle import sh3_color

F32 = np.float32
TILE = 16

# ---------------------------------------------------------------------------
# C part
# ---------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        from . import build as _b
        path = _b.library_path()
        if not os.path.exists(path):
            _b.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I = ctypes.c_int
        L.orc_blend_forward.argtypes = [I, I] + [P] * 14
        L.orc_blend_forward.restype = None
        L.orc_blend_backward.argtypes = [I, I] + [P] * 13
        L.orc_blend_backward.restype = None
        L.orc_brute_force.argtypes = [I, I, I] + [P] * 8 + [I] + [P] * 3
        L.orc_brute_force.restype = None
        L.orc_set_bands.argtypes = [ctypes.c_double] * 3
        L.orc_set_bands.restype = None
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = I
        L.orc_set_num_threads.argtypes = [I]
        L.orc_set_num_threads.restype = None
        _LIB = L
    return _LIB


def _p(a):
    """Address of a numpy array for a C call. The caller must hold a reference
    to `a` until the call returns (the address does not keep it alive)."""
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
# Eq. 1-2: SG colour
# ---------------------------------------------------------------------------

def sg_lobe(v, mu, s, a):
    """Eq. 1: G(v; mu, s, a) = a * exp(s (mu . v - 1)). v, mu: [..., 3]; s: [...]; a: [..., 3]."""
    return a * torch.exp(s * ((mu * v).sum(-1) - 1.0))[..., None]


def sg_color(c0, lobe_off, axis, sharp, amp, lmask, v):
    """Eq. 2 with per-lobe masks: c = c0 + sum_k m_k G(v; mu_k/|mu_k|, s_k, a_k).

    c0 [N,3], v [N,3] (unit), lobe_off [N+1] int, axis/amp [L,3], sharp/lmask [L].
    Returns the colour before the >= 0 clamp.
    """
    counts = np.diff(np.asarray(lobe_off))
    owner = torch.from_numpy(np.repeat(np.arange(len(counts)), counts))
    mu = axis / torch.linalg.norm(axis, dim=-1, keepdim=True)
    term = lmask[:, None] * sg_lobe(v[owner], mu, sharp, amp)
    return c0.index_add(0, owner, term)


# ---------------------------------------------------------------------------
# Binary32 decision recipe (identical order of operations on the GPU side)
# ---------------------------------------------------------------------------

@dataclass
class Decisions:
    visible: np.ndarray      # [N] bool
    radius: np.ndarray       # [N] int32 (0 when culled)
    rect: np.ndarray         # [N,4] int32 tile rectangle x0, y0, x1, y1 (half open)
    depth_bits: np.ndarray   # [N] uint32 bits of the binary32 camera-space depth
    xy32: np.ndarray         # [N,2] binary32 projected centre (reported only)
    conic32: np.ndarray      # [N,3] binary32 conic (reported only)
    touched: np.ndarray | None = None   # [N] int64 tiles of the 3-sigma rectangle (0 when culled)


def _clamp_tile(f, n):
    """floor'ed tile coordinate -> int in [0, n]; NaN -> 0."""
    out = np.zeros(f.shape, np.int64)
    ok = f > 0
    out[ok] = np.minimum(f[ok], n).astype(np.int64)
    out[f >= n] = n
    return out


def decisions_fp32(scene, cam) -> Decisions:
    """Cull / radius / tile rectangle / depth key in binary32, one rounding per
    operation in the written order, no fused multiply-add (the steps below are the recipe)."""
    with np.errstate(all="ignore"):
        p = scene.means.astype(F32)
        V = cam.viewmat.astype(F32)
        f = F32
        t = [((V[k, 0] * p[0] + V[k, 1] * p[1]) + V[k, 2] * p[2]) + V[k, 3] for k in range(3)]
        tz = t[2]
        near_ok = tz > f(cam.near)

        q = scene.quats.astype(F32)
        n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]
        r = f(1.0) / np.sqrt(n2)
        w, x, y, z = q[0] * r, q[1] * r, q[2] * r, q[3] * r
        one, two = f(1.0), f(2.0)
        R = [[one - two * (y * y + z * z), two * (x * y - w * z), two * (x * z + w * y)],
             [two * (x * y + w * z), one - two * (x * x + z * z), two * (y * z - w * x)],
             [two * (x * z - w * y), two * (y * z + w * x), one - two * (x * x + y * y)]]
        s = scene.scales.astype(F32)
        M = [[R[i][j] * s[j] for j in range(3)] for i in range(3)]
        S = {}
        for i in range(3):
            for j in range(i, 3):
                S[i, j] = (M[i][0] * M[j][0] + M[i][1] * M[j][1]) + M[i][2] * M[j][2]
                S[j, i] = S[i, j]

        fx, fy, cx, cy = f(cam.fx), f(cam.fy), f(cam.cx), f(cam.cy)
        tanx = (f(0.5) * f(cam.width)) / fx
        tany = (f(0.5) * f(cam.height)) / fy
        limx = f(1.3) * tanx
        limy = f(1.3) * tany
        ux = t[0] / tz
        uy = t[1] / tz
        ccx = np.minimum(limx, np.maximum(-limx, ux)) * tz
        ccy = np.minimum(limy, np.maximum(-limy, uy)) * tz
        tz2 = tz * tz
        j00 = fx / tz
        j11 = fy / tz
        j02 = -((fx * ccx) / tz2)
        j12 = -((fy * ccy) / tz2)
        A = [[j00 * V[0, j] + j02 * V[2, j] for j in range(3)],
             [j11 * V[1, j] + j12 * V[2, j] for j in range(3)]]
        B = [[(A[i][0] * S[0, j] + A[i][1] * S[1, j]) + A[i][2] * S[2, j] for j in range(3)]
             for i in range(2)]
        ca = ((B[0][0] * A[0][0] + B[0][1] * A[0][1]) + B[0][2] * A[0][2]) + f(0.3)
        cb = (B[0][0] * A[1][0] + B[0][1] * A[1][1]) + B[0][2] * A[1][2]
        cc = ((B[1][0] * A[1][0] + B[1][1] * A[1][1]) + B[1][2] * A[1][2]) + f(0.3)
        det = ca * cc - cb * cb
        det_ok = det > f(0.0)
        conA = cc / det
        conB = -(cb / det)
        conC = ca / det
        mid = f(0.5) * (ca + cc)
        lam1 = mid + np.sqrt(np.maximum(f(0.1), mid * mid - det))
        rf = np.ceil(f(3.0) * np.sqrt(lam1))
        px = (fx * ux + cx) - f(0.5)
        py = (fy * uy + cy) - f(0.5)
        sixteen, fifteen = f(16.0), f(15.0)
        tx0 = _clamp_tile(np.floor((px - rf) / sixteen), cam.tiles_x)
        tx1 = _clamp_tile(np.floor(((px + rf) + fifteen) / sixteen), cam.tiles_x)
        ty0 = _clamp_tile(np.floor((py - rf) / sixteen), cam.tiles_y)
        ty1 = _clamp_tile(np.floor(((py + rf) + fifteen) / sixteen), cam.tiles_y)
        area_ok = (tx1 > tx0) & (ty1 > ty0)
        opd = scene.gmask.astype(F32) * scene.opac.astype(F32)
        op_ok = opd >= f(1.0 / 255.0)
        finite = (np.isfinite(px) & np.isfinite(py) & np.isfinite(rf) & np.isfinite(conA)
                  & np.isfinite(conB) & np.isfinite(conC))
        vis = near_ok & det_ok & area_ok & op_ok & finite
        rad = np.where(vis, np.minimum(rf, f(2 ** 30)), 0).astype(np.int32)
        rect = np.stack([tx0, ty0, tx1, ty1], 1).astype(np.int32)
        rect[~vis] = 0
        depth_bits = tz.astype(F32).view(np.uint32).copy()
        dec = Decisions(vis, rad, rect, depth_bits,
                        np.stack([px, py], 1), np.stack([conA, conB, conC], 1))
        dec.touched = np.where(vis, (tx1 - tx0) * (ty1 - ty0), 0).astype(np.int64)
        return dec


# ---------------------------------------------------------------------------
# Duplicate, sort, ranges (tile lists)
# ---------------------------------------------------------------------------

def tile_lists(dec: Decisions, cam, tile_offset=0):
    """Pairs (tile, Gaussian) for every tile of every visible Gaussian's 3-sigma
    rectangle (the rule of the 3DGS rasterizer the paper keeps, Sec. 3.1 and
    Sec. 4), sorted by the 64-bit key (tile << 32 | depth bits), equal keys by
    Gaussian id.

    Returns keys [K] uint64, ids [K] int64, ranges [n_tiles, 2] int64.
    """
    ids_v = np.nonzero(dec.visible)[0]
    r = dec.rect[ids_v].astype(np.int64)
    h = r[:, 3] - r[:, 1]
    g = np.repeat(ids_v, h)
    start = np.repeat(np.cumsum(h) - h, h)
    ty = np.repeat(r[:, 1], h) + (np.arange(int(h.sum()), dtype=np.int64) - start)
    c0, c1 = dec.rect[g, 0].astype(np.int64), dec.rect[g, 2].astype(np.int64)
    cnt = c1 - c0
    K = int(cnt.sum())
    gid = np.repeat(g, cnt)
    start = np.repeat(np.cumsum(cnt) - cnt, cnt)
    tx = np.repeat(c0, cnt) + (np.arange(K, dtype=np.int64) - start)
    ty = np.repeat(ty, cnt)
    tile = tile_offset + ty * cam.tiles_x + tx
    keys = (tile.astype(np.uint64) << np.uint64(32)) | dec.depth_bits[gid].astype(np.uint64)
    order = np.lexsort((gid, keys))
    keys = keys[order]
    ids = gid[order]
    tiles_sorted = (keys >> np.uint64(32)).astype(np.int64) - tile_offset
    nt = cam.n_tiles
    starts = np.searchsorted(tiles_sorted, np.arange(nt), side="left")
    ends = np.searchsorted(tiles_sorted, np.arange(nt), side="right")
    ranges = np.stack([starts, ends], 1).astype(np.int64)
    return keys, ids.astype(np.int64), ranges


# ---------------------------------------------------------------------------
# FP64 projection and colour (differentiable with torch autograd)
# ---------------------------------------------------------------------------

PARAM_NAMES = ("means", "scales", "quats", "opac", "gmask", "c0", "axis", "sharp", "amp", "lmask")


def param_names(scene):
    """The differentiable inputs of a scene: the SG parameters, plus the SH
    coefficients when the scene uses the SH3 colour model."""
    return PARAM_NAMES + (("sh",) if getattr(scene, "sh", None) is not None else ())


def leaves(scene, requires_grad=True):
    """FP64 torch leaves, per-Gaussian rows: means [N,3] ... axis [L,3] ...
    sh [N,3,16] (from the stored [3][16][N])."""
    out = {}
    for k in param_names(scene):
        a = np.asarray(getattr(scene, k), np.float64)
        if a.ndim == 3:
            a = np.ascontiguousarray(a.transpose(2, 0, 1))
        else:
            a = a.T.copy() if a.ndim == 2 else a.copy()
        out[k] = torch.from_numpy(a).requires_grad_(requires_grad)
    return out


def quat_to_rot(q):
    """Rotation matrix of the normalised quaternion (w, x, y, z). q: [N,4] -> [N,3,3]."""
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)
    return R.reshape(-1, 3, 3)


def project_fp64(P, cam, vis_idx, lobe_off):
    """FP64 per-Gaussian projection for the visible subset.

    Returns xy [n,2], conic [n,3] (A, B, C), op [n] (o' = m_g o), rgb [n,3] (clamped >= 0).
    """
    idx = torch.from_numpy(vis_idx)
    Vm = torch.from_numpy(cam.viewmat.astype(np.float64))
    Rc, tc = Vm[:, :3], Vm[:, 3]
    mean = P["means"][idx]
    t = mean @ Rc.T + tc
    tx, ty, tz = t.unbind(-1)
    # Sigma_3D = R diag(s)^2 R^T
    R = quat_to_rot(P["quats"][idx])
    Ms = R * P["scales"][idx][:, None, :]
    Sig = Ms @ Ms.transpose(1, 2)
    # EWA: J (guard band 1.3 tan(fov/2)), Sigma_2D = J Rc Sigma Rc^T J^T + 0.3 I
    fx, fy = cam.fx, cam.fy
    limx = 1.3 * (0.5 * cam.width / fx)
    limy = 1.3 * (0.5 * cam.height / fy)
    ccx = torch.clamp(tx / tz, -limx, limx) * tz
    ccy = torch.clamp(ty / tz, -limy, limy) * tz
    zero = torch.zeros_like(tz)
    J = torch.stack([fx / tz, zero, -fx * ccx / (tz * tz),
                     zero, fy / tz, -fy * ccy / (tz * tz)], -1).reshape(-1, 2, 3)
    Amat = J @ Rc
    cov = Amat @ Sig @ Amat.transpose(1, 2)
    a = cov[:, 0, 0] + 0.3
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + 0.3
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], -1)
    x = fx * tx / tz + cam.cx - 0.5
    y = fy * ty / tz + cam.cy - 0.5
    xy = torch.stack([x, y], -1)
    op = P["gmask"][idx] * P["opac"][idx]
    # SG colour (Eq. 2) with view direction from the camera centre to the Gaussian
    cam_pos = -(Rc.T @ tc)
    d = mean - cam_pos
    v = d / torch.linalg.norm(d, dim=-1, keepdim=True)
    if "sh" in P:   # the SH3 baseline colour instead of the SG lobes
        return xy, conic, op, torch.clamp(sh3_color(P["sh"][idx], v), min=0.0)
    off = np.asarray(lobe_off, np.int64)
    counts = np.diff(off)[vis_idx]
    lobe_idx = _lobe_index_fast(off, vis_idx)
    sub_off = np.zeros(len(vis_idx) + 1, np.int64)
    np.cumsum(counts, out=sub_off[1:])
    li = torch.from_numpy(lobe_idx.astype(np.int64))
    col = sg_color(P["c0"][idx], sub_off, P["axis"][li], P["sharp"][li], P["amp"][li],
                   P["lmask"][li], v)
    rgb = torch.clamp(col, min=0.0)
    return xy, conic, op, rgb


def _lobe_index_fast(off, vis_idx):
    counts = np.diff(off)[vis_idx]
    starts = off[vis_idx]
    tot = int(counts.sum())
    base = np.repeat(starts - np.concatenate([[0], np.cumsum(counts)[:-1]]), counts)
    return base + np.arange(tot)


# ---------------------------------------------------------------------------
# Forward / backward of one view
# ---------------------------------------------------------------------------

@dataclass
class ViewResult:
    img: np.ndarray          # [3,H,W] f64
    T_final: np.ndarray      # [H,W] f64
    last: np.ndarray         # [H,W] int64 (position+1 inside the tile list)
    ambiguous: np.ndarray    # [H,W] bool
    sig: np.ndarray          # [H,W] uint64 hash of the contributing list positions
    dec: Decisions
    keys: np.ndarray
    ids: np.ndarray
    ranges: np.ndarray
    xy: np.ndarray           # [N,2] f64 (0 for culled)
    conic: np.ndarray        # [N,3]
    op: np.ndarray           # [N]
    rgb: np.ndarray          # [N,3]
    tile_sel: np.ndarray | None
    torch_state: tuple | None
    importance: np.ndarray | None = None   # [N] sum over pixels of alpha T (App. A.2)


def render_forward(scene, cam, tile_sel=None, need_grad=False):
    """One view. tile_sel: optional bool [n_tiles] -- render only those tiles."""
    dec = decisions_fp32(scene, cam)
    keys, ids, ranges = tile_lists(dec, cam)
    vis_idx = np.nonzero(dec.visible)[0]
    P = leaves(scene, requires_grad=need_grad)
    with torch.set_grad_enabled(need_grad):
        xy_t, con_t, op_t, rgb_t = project_fp64(P, cam, vis_idx, scene.lobe_off)
    N = scene.n
    xy = np.zeros((N, 2))
    con = np.zeros((N, 3))
    op = np.zeros(N)
    rgb = np.zeros((N, 3))
    xy[vis_idx] = xy_t.detach().numpy()
    con[vis_idx] = con_t.detach().numpy()
    op[vis_idx] = op_t.detach().numpy()
    rgb[vis_idx] = rgb_t.detach().numpy()
    H, W = cam.height, cam.width
    img = np.zeros((3, H, W))
    T = np.ones((H, W))
    last = np.zeros((H, W), np.int64)
    amb = np.zeros((H, W), np.uint8)
    sig = np.zeros((H, W), np.uint64)
    bg = _c(cam.bg, np.float64)
    sel = None if tile_sel is None else _c(tile_sel, np.uint8)
    weight = np.zeros(N)
    lib().orc_blend_forward(W, H, _p(ranges), _p(ids), _p(xy), _p(con), _p(op), _p(rgb),
                            _p(bg), _p(sel), _p(img), _p(T), _p(last), _p(amb), _p(sig),
                            _p(weight))
    state = (P, (xy_t, con_t, op_t, rgb_t), vis_idx) if need_grad else None
    return ViewResult(img, T, last, amb.astype(bool), sig, dec, keys, ids, ranges,
                      xy, con, op, rgb, sel, state, weight)


def render_backward(res: ViewResult, scene, cam, dimg):
    """Gradients of L = sum(dimg * img) w.r.t. every float input (FP64 numpy,
    same layout as the scene arrays: [3][N], [N], [3][L], ...)."""
    assert res.torch_state is not None, "render_forward(..., need_grad=True) first"
    P, outs, vis_idx = res.torch_state
    N = scene.n
    dxy = np.zeros((N, 2))
    dcon = np.zeros((N, 3))
    dop = np.zeros(N)
    drgb = np.zeros((N, 3))
    bg = _c(cam.bg, np.float64)
    dimg64 = _c(dimg, np.float64)   # keep the converted copy alive across the call
    lib().orc_blend_backward(cam.width, cam.height, _p(res.ranges), _p(res.ids), _p(res.xy),
                             _p(res.conic), _p(res.op), _p(res.rgb), _p(bg), _p(res.tile_sel),
                             _p(dimg64), _p(dxy), _p(dcon), _p(dop), _p(drgb))
    grads_out = [torch.from_numpy(a[vis_idx]) for a in (dxy, dcon, dop, drgb)]
    names = param_names(scene)
    leaves_ = [P[k] for k in names]
    gl = torch.autograd.grad(list(outs), leaves_, grad_outputs=grads_out, allow_unused=True)
    out = {}
    for k, g in zip(names, gl):
        ref = getattr(scene, k)
        if g is None:
            out[k] = np.zeros(ref.shape)
        else:
            g = g.numpy()
            if g.ndim == 3:
                out[k] = np.ascontiguousarray(g.transpose(1, 2, 0))
            else:
                out[k] = g.T.copy() if g.ndim == 2 else g.copy()
    return out


def render(scene, cams, dimgs=None, tile_sel=None):
    """Several views of one scene. Returns per-view ViewResults and, when dimgs
    is given, the gradients summed over the views."""
    results, grads = [], None
    for i, cam in enumerate(cams):
        sel = None if tile_sel is None else tile_sel[i]
        r = render_forward(scene, cam, sel, need_grad=dimgs is not None)
        results.append(r)
        if dimgs is not None:
            g = render_backward(r, scene, cam, dimgs[i])
            grads = g if grads is None else {k: grads[k] + g[k] for k in g}
    return results, grads


def brute_force(scene, cam, gate=True):
    """Per-pixel walk over all visible Gaussians in global (depth key, id) order."""
    dec = decisions_fp32(scene, cam)
    vis_idx = np.nonzero(dec.visible)[0]
    P = leaves(scene, requires_grad=False)
    with torch.no_grad():
        xy_t, con_t, op_t, rgb_t = project_fp64(P, cam, vis_idx, scene.lobe_off)
    N = scene.n
    xy = np.zeros((N, 2))
    con = np.zeros((N, 3))
    op = np.zeros(N)
    rgb = np.zeros((N, 3))
    xy[vis_idx] = xy_t.numpy()
    con[vis_idx] = con_t.numpy()
    op[vis_idx] = op_t.numpy()
    rgb[vis_idx] = rgb_t.numpy()
    H, W = cam.height, cam.width
    img = np.zeros((3, H, W))
    T = np.ones((H, W))
    last = np.zeros((H, W), np.int64)
    # converted copies are bound to names so they outlive the C call
    depth_bits = _c(dec.depth_bits, np.uint32)
    rect = _c(dec.rect, np.int32)
    vis = _c(dec.visible, np.uint8)
    bg = _c(cam.bg, np.float64)
    lib().orc_brute_force(N, W, H, _p(depth_bits), _p(rect), _p(vis), _p(xy), _p(con), _p(op),
                          _p(rgb), _p(bg), int(gate), _p(img), _p(T), _p(last))
    return img, T, last


def set_bands(alpha=2e-5, T=5e-5, power=1e-6):
    lib().orc_set_bands(alpha, T, power)


def num_threads():
    return int(lib().orc_num_threads())


def set_num_threads(n):
    """Threads of the C blend loops (OpenMP) from now on."""
    lib().orc_set_num_threads(int(n))
