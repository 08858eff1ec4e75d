"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(Eq. 1, 2, 10, 12; the EWA projection of an isotropic Gaussian), invariants of
front-to-back compositing (Sec. 3.1), brute force over all depth-sorted
Gaussians, a pure-Python tile binning loop, and FP64 central differences.
"""
import math

import numpy as np
import pytest
import torch

from paper_2509_07021_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def one_gaussian_scene(mean, scale, quat=(1, 0, 0, 0), opac=0.8, c0=(0.2, 0.5, 0.9),
                       lobes=(), gmask=1.0):
    n_l = len(lobes)
    f = np.float32
    axis = np.array([l[0] for l in lobes], f).T.reshape(3, n_l)
    sharp = np.array([l[1] for l in lobes], f).reshape(n_l)
    amp = np.array([l[2] for l in lobes], f).T.reshape(3, n_l)
    lmask = np.array([l[3] if len(l) > 3 else 1.0 for l in lobes], f).reshape(n_l)
    return synth.Scene(
        means=np.array(mean, f).reshape(3, 1), scales=np.array(scale, f).reshape(3, 1),
        quats=np.array(quat, f).reshape(4, 1), opac=np.array([opac], f),
        gmask=np.array([gmask], f), c0=np.array(c0, f).reshape(3, 1),
        lobe_off=np.array([0, n_l], np.int32), axis=axis, sharp=sharp, amp=amp, lmask=lmask)


def concat(scenes):
    offs = [0]
    for s in scenes:
        offs.append(offs[-1] + s.n_lobes)
    lo = np.concatenate([[0]] + [s.lobe_off[1:] + o for s, o in zip(scenes, offs)]).astype(np.int32)
    kw = {}
    for k in synth.Scene.FLOAT_FIELDS:
        kw[k] = np.concatenate([getattr(s, k) for s in scenes], axis=-1)
    return synth.Scene(lobe_off=lo, **kw)


def t64(a):
    return torch.tensor(np.asarray(a, np.float64))


def f32(x):
    """The value a binary32 scene array holds for x."""
    return float(np.float32(x))


# ---------------------------------------------------------------------------
# Eq. 1-2, Eq. 10, Eq. 12
# ---------------------------------------------------------------------------

def _single_lobe_color(orc, v, mu, s, a, c0=(0.0, 0.0, 0.0), m=1.0):
    v = np.atleast_2d(np.asarray(v, np.float64))
    n = v.shape[0]
    c0 = t64(np.tile(np.asarray(c0, np.float64), (n, 1)))
    off = np.arange(n + 1)
    axis = t64(np.tile(mu, (n, 1)))
    return orc.sg_color(c0, off, axis, t64(np.full(n, s)), t64(np.tile(a, (n, 1))),
                        t64(np.full(n, m)), t64(v)).numpy()


def test_sg_value_on_axis_and_antipode(orc):
    """Eq. 1 and Eq. 10: the lobe is a on its axis and a e^{-2s} at the antipode."""
    rng = np.random.default_rng(0)
    for _ in range(10):
        mu = rng.standard_normal(3)
        mu_hat = mu / np.linalg.norm(mu)
        s = float(rng.uniform(0.1, 60))
        a = rng.normal(0, 1, 3)
        c0 = rng.random(3)
        on = _single_lobe_color(orc, mu_hat, mu, s, a, c0)[0]
        anti = _single_lobe_color(orc, -mu_hat, mu, s, a, c0)[0]
        np.testing.assert_allclose(on, c0 + a, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(anti, c0 + a * math.exp(-2 * s), rtol=1e-12, atol=1e-14)
        # Eq. 10: dynamic range over v equals |a|(1 - e^{-2s}) per channel
        np.testing.assert_allclose(np.abs(on - anti), np.abs(a) * (1 - math.exp(-2 * s)),
                                   rtol=1e-12)


def test_sg_degenerate_cases(orc):
    """s = 0 makes the lobe the constant a; m_l = 0 removes it; no lobes leaves c0."""
    rng = np.random.default_rng(1)
    v = rng.standard_normal((7, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    a = np.array([0.3, -0.2, 0.7])
    c0 = np.array([0.1, 0.2, 0.3])
    col = _single_lobe_color(orc, v, (0.0, 0.0, 1.0), 0.0, a, c0)
    np.testing.assert_allclose(col, np.tile(c0 + a, (7, 1)), rtol=1e-15)
    col = _single_lobe_color(orc, v, (0.0, 0.0, 1.0), 5.0, a, c0, m=0.0)
    np.testing.assert_allclose(col, np.tile(c0, (7, 1)), rtol=0, atol=0)
    n = 5
    out = orc.sg_color(t64(np.tile(c0, (n, 1))), np.zeros(n + 1, np.int64),
                       t64(np.zeros((0, 3))), t64(np.zeros(0)), t64(np.zeros((0, 3))),
                       t64(np.zeros(0)), t64(v[:n])).numpy()
    np.testing.assert_array_equal(out, np.tile(c0, (n, 1)))


def test_sg_sphere_integral_and_compensation(orc):
    """Appendix derivation: the lobe integrates to 2 pi a (1 - e^{-2s}) / s over S^2,
    so Eq. 12's compensation is its mean, a (1 - e^{-2s}) / (2s)."""
    rng = np.random.default_rng(2)
    nu, nphi = 400, 64
    u, wu = np.polynomial.legendre.leggauss(nu)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    U, PHI = np.meshgrid(u, phi, indexing="ij")
    sinth = np.sqrt(1 - U ** 2)
    local = np.stack([sinth * np.cos(PHI), sinth * np.sin(PHI), U], -1).reshape(-1, 3)
    wts = (wu[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    for s in (0.5, 1.0, 7.3, 25.0):
        mu = rng.standard_normal(3)
        mu /= np.linalg.norm(mu)
        # orthonormal frame with mu as the z axis
        e1 = np.cross(mu, [1.0, 0.0, 0.0] if abs(mu[0]) < 0.9 else [0.0, 1.0, 0.0])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(mu, e1)
        v = local @ np.stack([e1, e2, mu])
        a = rng.normal(0, 1, 3)
        col = _single_lobe_color(orc, v, mu, s, a)
        integral = (col * wts[:, None]).sum(0)
        expect = 2 * np.pi * a * (1 - math.exp(-2 * s)) / s
        np.testing.assert_allclose(integral, expect, rtol=1e-9)
        np.testing.assert_allclose(integral / (4 * np.pi), a * (1 - math.exp(-2 * s)) / (2 * s),
                                   rtol=1e-9)


def test_golden_closed_forms(orc):
    """Fixture tests/golden/sg_closed_forms.txt (Eq. 1, Eq. 10, Eq. 12)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "sg_closed_forms.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 4
    for s, a, vmax, vmin, dc0 in ((float(x) for x in r) for r in rows):
        mu = np.array([0.0, 0.6, 0.8])
        on = _single_lobe_color(orc, mu, mu, s, (a, a, a))[0, 0]
        anti = _single_lobe_color(orc, -mu, mu, s, (a, a, a))[0, 0]
        assert on == pytest.approx(vmax, rel=1e-12)
        assert anti == pytest.approx(vmin, rel=1e-12, abs=1e-300)
        assert a * (1 - math.exp(-2 * s)) / (2 * s) == pytest.approx(dc0, rel=1e-12)


def test_golden_parameter_counts():
    """Eq. 3 and Table 3: rho_o = 11 base floats per Gaussian, rho_s = 7 per lobe,
    3 + 7 n colour floats (24 for three lobes, 48 for degree-3 SH)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "param_counts.txt")
    vals = dict(l.split()[:2] for l in open(path) if l.strip() and not l.startswith("#"))
    scene = synth.make_scene(np.random.default_rng(0), 10, lobes=3)
    per_g = sum(getattr(scene, k).shape[0] for k in ("means", "scales", "quats")) + 1
    per_l = sum(getattr(scene, k).shape[0] for k in ("axis", "amp")) + 1
    assert per_g == int(vals["rho_o"])
    assert per_l == int(vals["rho_s"])
    assert scene.c0.shape[0] + 3 * per_l == int(vals["colour_3_lobes"])


# ---------------------------------------------------------------------------
# EWA projection (Sec. 3.1) in closed form
# ---------------------------------------------------------------------------

def _proj(orc, scene, cam):
    P = orc.leaves(scene, requires_grad=False)
    vis = np.arange(scene.n)
    xy, con, op, rgb = orc.project_fp64(P, cam, vis, scene.lobe_off)
    return xy.numpy(), con.numpy(), op.numpy(), rgb.numpy()


def _cov_from_conic(con):
    A, B, C = con
    M = np.linalg.inv(np.array([[A, B], [B, C]]))
    return M


def test_ewa_isotropic_on_axis(orc):
    f, z, sig = 150.0, 4.0, 0.05
    rng = np.random.default_rng(3)
    q = rng.standard_normal(4)
    scene = one_gaussian_scene((0, 0, z), (sig, sig, sig), quat=q)
    cam = synth.make_camera(128, 128, f)
    xy, con, _, _ = _proj(orc, scene, cam)
    s2 = f * f * sig * sig / (z * z) + 0.3
    np.testing.assert_allclose(_cov_from_conic(con[0]), np.diag([s2, s2]), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(xy[0], [63.5, 63.5], rtol=0, atol=1e-12)
    dec = orc.decisions_fp32(scene, cam)
    # isotropic: mid^2 - det = 0, so the inherited floor max(0.1, .) sets lambda_1 = s2 + sqrt(0.1)
    assert dec.radius[0] == math.ceil(3 * math.sqrt(s2 + math.sqrt(0.1)))


def test_ewa_quaternion_convention(orc):
    """q = (w, x, y, z): 90 deg about x swaps the y and z scales; theta about z gives
    off-diagonal f^2/z^2 (sx^2 - sy^2) sin(theta) cos(theta)."""
    f, z = 150.0, 4.0
    sx, sy, sz = 0.02, 0.05, 0.11
    c = math.cos(math.pi / 4)
    scene = one_gaussian_scene((0, 0, z), (sx, sy, sz), quat=(c, c, 0, 0))
    cam = synth.make_camera(128, 128, f)
    _, con, _, _ = _proj(orc, scene, cam)
    k = f * f / (z * z)
    np.testing.assert_allclose(_cov_from_conic(con[0]),
                               np.diag([k * sx * sx + 0.3, k * sz * sz + 0.3]), rtol=1e-6,
                               atol=1e-9)
    th = 0.7
    scene = one_gaussian_scene((0, 0, z), (sx, sy, sz),
                               quat=(math.cos(th / 2), 0, 0, math.sin(th / 2)))
    _, con, _, _ = _proj(orc, scene, cam)
    cs, sn = math.cos(th), math.sin(th)
    expect = k * np.array([[cs * cs * sx * sx + sn * sn * sy * sy, cs * sn * (sx * sx - sy * sy)],
                           [cs * sn * (sx * sx - sy * sy), sn * sn * sx * sx + cs * cs * sy * sy]])
    np.testing.assert_allclose(_cov_from_conic(con[0]), expect + 0.3 * np.eye(2), rtol=1e-6)


@pytest.mark.parametrize("X", [0.7, 3.9, -5.5])
def test_ewa_off_axis(orc, X):
    """Gaussian at (X, 0, Z): J = [[f/Z, 0, -f X'/Z^2], [0, f/Z, 0]] with X'/Z clamped to
    1.3 tan(fov_x / 2)."""
    f, Z, sig = 150.0, 4.0, 0.03
    W = 128
    scene = one_gaussian_scene((X, 0, Z), (sig, sig, sig))
    cam = synth.make_camera(W, 128, f)
    xy, con, _, _ = _proj(orc, scene, cam)
    X, sig = float(np.float32(X)), float(np.float32(sig))  # the scene stores binary32
    lim = 1.3 * (W / 2) / f
    u = max(-lim, min(lim, X / Z))
    a = sig * sig * (f * f / Z ** 2 + f * f * u * u / Z ** 2) + 0.3
    c = sig * sig * f * f / Z ** 2 + 0.3
    np.testing.assert_allclose(_cov_from_conic(con[0]), np.diag([a, c]), rtol=1e-6, atol=1e-9)
    assert xy[0, 0] == pytest.approx(f * X / Z + 64 - 0.5, abs=1e-12)


def test_view_direction_and_camera_pose(orc):
    """Colour uses v = (p - cam)/|p - cam| (camera centre -R^T t), checked with a lobe
    whose axis equals v (colour c0 + a) and one pointing away (c0 + a e^{-2s})."""
    eye = np.array([1.0, -2.0, -6.0])
    p = np.array([0.3, 0.4, 0.5])
    V = synth.look_at(eye, p + np.array([0.1, 0.0, 0.0]))
    cam = synth.make_camera(256, 256, 200.0, viewmat=V)
    v = (p - eye) / np.linalg.norm(p - eye)
    s, a = 9.0, np.array([0.3, 0.6, 0.9])
    for sign, expect in ((1, a), (-1, a * math.exp(-2 * s))):
        scene = one_gaussian_scene(p, (0.05,) * 3, c0=(0.1, 0.1, 0.1),
                                   lobes=[(tuple(sign * v), s, tuple(a))])
        _, _, _, rgb = _proj(orc, scene, cam)
        # binary32 storage of the scene bounds the agreement
        np.testing.assert_allclose(rgb[0], 0.1 + expect, rtol=2e-5, atol=2e-6)


# ---------------------------------------------------------------------------
# Compositing (Sec. 3.1) in closed form and invariants
# ---------------------------------------------------------------------------

def _rect_fp64(x, r, n):
    lo = math.floor((x - r) / 16)
    hi = math.floor((x + r + 15) / 16)
    return max(0, min(n, lo)), max(0, min(n, hi))


def test_single_gaussian_image(orc):
    f, z, sig, o = 150.0, 4.0, 0.06, 0.7
    W = H = 64
    cam = synth.make_camera(W, H, f, bg=(0.05, 0.1, 0.2))
    scene = one_gaussian_scene((0.1, -0.05, z), (sig,) * 3, opac=o, c0=(0.2, 0.5, 0.9))
    res = orc.render_forward(scene, cam)
    sig, o, X, Y = f32(sig), f32(o), f32(0.1), f32(-0.05)
    # isotropic Sigma_3D = sig^2 I: Sigma_2D = sig^2 J J^T + 0.3 I
    J = np.array([[f / z, 0, -f * X / z ** 2], [0, f / z, -f * Y / z ** 2]])
    cov = sig * sig * J @ J.T + 0.3 * np.eye(2)
    Q = np.linalg.inv(cov)
    x0 = f * X / z + W / 2 - 0.5
    y0 = f * Y / z + H / 2 - 0.5
    mid = 0.5 * (cov[0, 0] + cov[1, 1])
    lam = mid + math.sqrt(max(0.1, mid * mid - np.linalg.det(cov)))
    r = math.ceil(3 * math.sqrt(lam))
    tx = _rect_fp64(x0, r, 4)
    ty = _rect_fp64(y0, r, 4)
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    dx, dy = ii - x0, jj - y0
    q = Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy
    al = np.minimum(0.99, o * np.exp(-0.5 * q))
    inside = ((ii // 16 >= tx[0]) & (ii // 16 < tx[1]) & (jj // 16 >= ty[0]) & (jj // 16 < ty[1]))
    al = np.where(inside & (al >= 1 / 255), al, 0.0)
    for ch, (c, b) in enumerate(zip((0.2, 0.5, 0.9), (0.05, 0.1, 0.2))):
        np.testing.assert_allclose(res.img[ch], f32(c) * al + f32(b) * (1 - al), atol=1e-12)
    np.testing.assert_allclose(res.T_final, 1 - al, atol=1e-12)
    np.testing.assert_array_equal(res.last, (al > 0).astype(np.int64))


def test_two_gaussians_composite(orc):
    """c1 a1 + c2 a2 (1 - a1), front to back by depth; swapping depths swaps the order."""
    f, W = 150.0, 32
    cam = synth.make_camera(W, W, f)
    g1 = one_gaussian_scene((0, 0, 3.0), (0.03,) * 3, opac=0.6, c0=(1, 0, 0))
    g2 = one_gaussian_scene((0, 0, 5.0), (0.05,) * 3, opac=0.5, c0=(0, 0, 1))
    res = orc.render_forward(concat([g1, g2]), cam)
    res_sw = orc.render_forward(concat([g2, g1]), cam)
    np.testing.assert_array_equal(res.img, res_sw.img)
    s2 = [f * f * f32(0.03) ** 2 / 9 + 0.3, f * f * f32(0.05) ** 2 / 25 + 0.3]
    jj, ii = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    d2 = (ii - 15.5) ** 2 + (jj - 15.5) ** 2
    a1 = f32(0.6) * np.exp(-0.5 * d2 / s2[0])
    a2 = f32(0.5) * np.exp(-0.5 * d2 / s2[1])
    a1 = np.where(a1 >= 1 / 255, a1, 0)
    a2 = np.where(a2 >= 1 / 255, a2, 0)
    np.testing.assert_allclose(res.img[0], a1, atol=1e-12)
    np.testing.assert_allclose(res.img[2], a2 * (1 - a1), atol=1e-12)
    np.testing.assert_allclose(res.T_final, (1 - a1) * (1 - a2), atol=1e-12)


def test_alpha_rules(orc):
    """0.99 clamp, 1/255 skip and the 1e-4 stop (which does not blend the stopping pair)."""
    f, W = 150.0, 16
    cam = synth.make_camera(W, W, f)
    # opacity above 0.99 at the centre is clamped to 0.99
    g = one_gaussian_scene((0, 0, 4.0), (0.2,) * 3, opac=0.999, c0=(1, 1, 1))
    res = orc.render_forward(g, cam)
    assert res.T_final.min() == pytest.approx(0.01, rel=1e-12)
    # opacity below 1/255 is culled, image empty
    g = one_gaussian_scene((0, 0, 4.0), (0.2,) * 3, opac=0.0035, c0=(1, 1, 1))
    res = orc.render_forward(g, cam)
    assert res.img.max() == 0.0 and res.last.max() == 0
    # two big clamped Gaussians give T = 1e-4 exactly -> the second would reach 1e-4 which
    # is not below the stop, so it blends; a third would give 1e-6 < 1e-4 -> stop, not blended
    gs = [one_gaussian_scene((0, 0, 4.0 + i), (0.5 * (4.0 + i) / 4,) * 3, opac=1.0,
                             c0=(1, 1, 1)) for i in range(3)]
    res = orc.render_forward(concat(gs), cam)
    c = res.img[0]
    # pixels where all three reach the clamp: T after two = 1e-4 (float rounding either way)
    centre = res.last[7, 7]
    assert centre in (1, 2)
    if centre == 2:
        assert res.T_final[7, 7] == pytest.approx(1e-4, rel=1e-9)
        assert c[7, 7] == pytest.approx(0.9999, rel=1e-9)


def test_weight_sum_and_monotone_T(orc):
    """With every colour 1 and a black background, sum_i alpha_i T_i = 1 - T_final."""
    rng = np.random.default_rng(5)
    scene = synth.make_scene(rng, 400, lobes=2, means="cube", masks="uniform")
    scene.c0[:] = 1.0
    scene.lmask[:] = 0.0
    cam = synth.make_camera(96, 80, 120.0)
    res = orc.render_forward(scene, cam)
    for ch in range(3):
        np.testing.assert_allclose(res.img[ch], 1 - res.T_final, atol=1e-12)
    assert (res.T_final >= 1e-4).all() and (res.T_final <= 1).all()
    lens = res.ranges[:, 1] - res.ranges[:, 0]
    ty, tx = np.meshgrid(np.arange(80) // 16, np.arange(96) // 16, indexing="ij")
    assert (res.last <= lens[ty * cam.tiles_x + tx]).all()
    assert res.last.max() > 3
    # T is non-increasing as more of the list is walked: truncating every tile list
    # to its first k entries can only raise T_final
    prev = None
    for k in (1, 3, 10, 10 ** 6):
        r = res.ranges.copy()
        r[:, 1] = np.minimum(r[:, 1], r[:, 0] + k)
        img = np.zeros((3, 80, 96))
        T = np.ones((80, 96))
        last = np.zeros((80, 96), np.int64)
        amb = np.zeros((80, 96), np.uint8)
        p = orc.sg_oracle._p
        bg = np.zeros(3)
        orc.lib().orc_blend_forward(96, 80, p(r), p(res.ids), p(res.xy), p(res.conic),
                                    p(res.op), p(res.rgb), p(bg), None, p(img), p(T),
                                    p(last), p(amb), None, None)
        if prev is not None:
            assert (T <= prev + 1e-15).all()
        prev = T
    np.testing.assert_array_equal(prev, res.T_final)


def test_mask_readings(orc):
    """m_g multiplies opacity and m_l multiplies the whole lobe term."""
    rng = np.random.default_rng(6)
    scene = synth.make_scene(rng, 200, lobes=3, means="cube", masks="uniform")
    cam = synth.make_camera(64, 64, 80.0)
    ref = orc.render_forward(scene, cam)
    s2 = scene.copy()
    s2.opac = (scene.opac.astype(np.float64) * scene.gmask).astype(np.float32)
    s2.gmask[:] = 1.0
    s2.amp = scene.amp * scene.lmask[None, :]
    s2.lmask[:] = 1.0
    res = orc.render_forward(s2, cam)
    # the products are rounded to binary32 once, hence a small tolerance
    np.testing.assert_allclose(res.img, ref.img, atol=5e-6)


# ---------------------------------------------------------------------------
# Tiling and sorting
# ---------------------------------------------------------------------------

def test_tile_lists_match_python_loop(orc):
    """The oracle's lists against a plain loop over the rule of the rasterizer
    the paper keeps: tile t's list holds every visible Gaussian whose 3-sigma
    rectangle contains t, in ascending (depth bits, index) order."""
    rng = np.random.default_rng(7)
    scene = synth.make_scene(rng, 150, lobes=1, means="cube", masks="uniform")
    cam = synth.make_camera(70, 50, 70.0)
    dec = orc.decisions_fp32(scene, cam)
    keys, ids, ranges = orc.tile_lists(dec, cam)
    total = 0
    for t in range(cam.n_tiles):
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        members = [g for g in range(scene.n) if dec.visible[g]
                   and dec.rect[g, 0] <= tx < dec.rect[g, 2] and dec.rect[g, 1] <= ty < dec.rect[g, 3]]
        members.sort(key=lambda g: (int(dec.depth_bits[g]), g))
        got = ids[ranges[t, 0]:ranges[t, 1]].tolist()
        assert got == members, t
        assert all(int(k) >> 32 == t for k in keys[ranges[t, 0]:ranges[t, 1]])
        total += len(members)
    assert ranges[-1, 1] == len(ids) == total
    np.testing.assert_array_equal(dec.touched, np.bincount(ids, minlength=scene.n))
    rect_area = (dec.rect[:, 2] - dec.rect[:, 0]) * (dec.rect[:, 3] - dec.rect[:, 1])
    np.testing.assert_array_equal(dec.touched, np.where(dec.visible, rect_area, 0))


@pytest.mark.parametrize("seed", [0, 1])
def test_library_binning_leaves_out_only_unreachable_tiles(orc, seed):
    """The library's tighter binning (restated in tight_binning) keeps an
    ordered sub-list of the oracle's lists, every pair it leaves out has
    q > 2 ln(255 o') on its whole tile in FP64 (alpha below 1/255 at every
    pixel, so the blend skips it there), and every pair it keeps is reachable
    or within the bound's enlargement."""
    from parity_util import box_min_q, unreachable
    import tight_binning
    rng = np.random.default_rng(300 + seed)
    scene = synth.make_scene(rng, 3000, lobes=1, means="cube", cube_side=1.5, masks="uniform")
    scene.scales *= np.exp(rng.normal(0.0, 0.7, scene.scales.shape)).astype(np.float32)  # anisotropic
    cam = synth.make_camera(200, 150, 180.0)
    res = orc.render_forward(scene, cam)
    dec = res.dec
    bound = tight_binning.binning_bound(scene)
    keep = tight_binning.kept_pairs(dec, bound, cam, res.keys, res.ids)
    tiles = (res.keys >> np.uint64(32)).astype(np.int64)
    assert 0 < keep.sum() < 0.9 * len(keep)
    assert unreachable(res, cam, tiles[~keep], res.ids[~keep]).all()
    g = res.ids[keep]
    qk = box_min_q(res.conic[g], res.xy[g], tiles[keep] % cam.tiles_x, tiles[keep] // cam.tiles_x)
    assert np.all(qk <= 1.02 * 2.0 * np.log(255.0 * res.op[g]) + 0.5)
    np.testing.assert_array_equal(tight_binning.touched(dec, bound), np.bincount(g, minlength=scene.n))


def test_log2_recipe_accuracy():
    """The library's binning log2 (atanh series on the mantissa) against FP64 log2 over the
    range 255 o' takes: the series stops at s^7 with s <= 1/3, so the error is at
    most (2 / ln 2) s^9 / (9 (1 - s^2)) = 1.8e-5 (plus binary32 rounding); exact at
    powers of two."""
    from tight_binning import log2_recipe
    x = np.concatenate([np.geomspace(1.0, 255.0, 4001), 2.0 ** np.arange(0, 8)]).astype(np.float32)
    got = log2_recipe(x).astype(np.float64)
    ref = np.log2(x.astype(np.float64))
    bound = 2.0 / np.log(2.0) * (1 / 3) ** 9 / (9 * (1 - 1 / 9)) + 2e-6
    assert np.all(np.abs(got - ref) <= bound)
    np.testing.assert_array_equal(log2_recipe(np.float32(2.0) ** np.arange(0, 8).astype(np.float32)),
                                  np.arange(0, 8).astype(np.float32))


def test_rect_matches_fp64_away_from_boundaries(orc):
    """The binary32 decisions agree with FP64 arithmetic wherever FP64 is not
    within a relative 1e-5 of a rounding boundary."""
    rng = np.random.default_rng(8)
    scene = synth.make_scene(rng, 3000, lobes=0, means="cube", masks="uniform")
    cam = synth.make_camera(128, 128, 150.0)
    dec = orc.decisions_fp32(scene, cam)
    P = orc.leaves(scene, requires_grad=False)
    vis = np.nonzero(dec.visible)[0]
    xy, con, op, _ = orc.project_fp64(P, cam, vis, scene.lobe_off)
    xy, con = xy.numpy(), con.numpy()
    cov = np.linalg.inv(np.stack([np.stack([con[:, 0], con[:, 1]], -1),
                                  np.stack([con[:, 1], con[:, 2]], -1)], -2))
    a, b, c = cov[:, 0, 0], cov[:, 0, 1], cov[:, 1, 1]
    mid = 0.5 * (a + c)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - (a * c - b * b)))
    r64 = 3 * np.sqrt(lam)
    safe = np.abs(r64 - np.round(r64)) > 1e-4 * r64
    assert safe.mean() > 0.99
    np.testing.assert_array_equal(dec.radius[vis][safe], np.ceil(r64[safe]).astype(np.int32))
    np.testing.assert_allclose(dec.xy32[vis], xy, rtol=1e-6, atol=1e-4)


def test_depth_keys_and_conic_against_fp64(orc):
    """The binary32 recipe's depth t_z = ((V20 px + V21 py) + V22 pz) + V23 lies within
    the forward error bound of a 4-term dot product, gamma_4 sum |terms|, of the FP64
    depth; any pair the binary32 keys order differently from FP64 depth lies within
    the two bounds of each other (near-equal depths only). The binary32 conic stays
    within a relative 1e-5 of the FP64 projection's."""
    rng = np.random.default_rng(9)
    scene = synth.make_scene(rng, 4000, lobes=0, means="cube", cube_side=2.0, masks="uniform")
    cam = synth.make_camera(160, 120, 150.0, viewmat=synth.look_at((0.7, -0.4, 0.3), (0.1, 0.2, 4.0)))
    dec = orc.decisions_fp32(scene, cam)
    vis = np.nonzero(dec.visible)[0]
    assert len(vis) > 3000
    z32 = dec.depth_bits[vis].view(np.float32).astype(np.float64)
    V = np.asarray(cam.viewmat, np.float32).astype(np.float64)
    p = scene.means.astype(np.float64)[:, vis]
    terms = np.stack([V[2, 0] * p[0], V[2, 1] * p[1], V[2, 2] * p[2], np.full(len(vis), V[2, 3])])
    z64 = terms.sum(0)
    u = 2.0 ** -24
    bound = 4 * u / (1 - 4 * u) * np.abs(terms).sum(0)
    assert np.all(np.abs(z32 - z64) <= bound)
    # order of the keys (ties by index, as the stable sort) against FP64 depth
    order = np.lexsort((vis, dec.depth_bits[vis]))
    zs, bs = z64[order], bound[order]
    i, j = np.triu_indices(len(zs), 1)
    inverted = zs[j] < zs[i]
    assert inverted.sum() <= 10
    assert np.all(zs[i][inverted] - zs[j][inverted] <= bs[i][inverted] + bs[j][inverted])
    P = orc.leaves(scene, requires_grad=False)
    _, con, _, _ = orc.project_fp64(P, cam, vis, scene.lobe_off)
    con = con.numpy()
    nrm = np.sqrt(con[:, 0] ** 2 + 2 * con[:, 1] ** 2 + con[:, 2] ** 2)
    assert (np.abs(dec.conic32[vis].astype(np.float64) - con).max(1) / nrm).max() < 1e-5


def test_tiled_equals_brute_force(orc):
    for seed in range(3):
        rng = np.random.default_rng(100 + seed)
        scene = synth.make_scene(rng, 64, lobes=synth.LOBE_MIX, means="cube", masks="uniform")
        cam = synth.make_camera(32, 32, 40.0, bg=rng.random(3))
        res = orc.render_forward(scene, cam)
        img, T, last = orc.brute_force(scene, cam, gate=True)
        np.testing.assert_array_equal(res.img, img)
        np.testing.assert_array_equal(res.T_final, T)
        # positions in the 3-sigma gated (depth, index) order are those of the tile lists
        np.testing.assert_array_equal(res.last, last)
        assert res.last.max() > 0


def test_footprint_cutoff_is_small(orc):
    """Dropping the 3-sigma tile gate changes the image only by the tails beyond it."""
    rng = np.random.default_rng(9)
    scene = synth.make_scene(rng, 64, lobes=1, means="cube", masks="uniform")
    cam = synth.make_camera(32, 32, 40.0)
    img_g, _, _ = orc.brute_force(scene, cam, gate=True)
    img_f, _, _ = orc.brute_force(scene, cam, gate=False)
    assert np.abs(img_g - img_f).max() < 0.05


# ---------------------------------------------------------------------------
# Adjoint vs FP64 central finite differences
# ---------------------------------------------------------------------------

def _fd_scene(seed):
    rng = np.random.default_rng(seed)
    scene = synth.make_scene(rng, 14, lobes=synth.LOBE_MIX, means="cube", masks="uniform")
    scene.scales *= 3.0
    cam = synth.make_camera(40, 36, 45.0, bg=(0.3, 0.1, 0.6))
    dimg = rng.normal(0, 1, (3, cam.height, cam.width))
    return scene, cam, dimg


def _loss(orc, scene, cam, dimg):
    res = orc.render_forward(scene, cam)
    return float((res.img * dimg).sum()), res


def _same_decisions(r0, r1):
    return (np.array_equal(r0.dec.visible, r1.dec.visible) and np.array_equal(r0.dec.rect, r1.dec.rect)
            and np.array_equal(r0.ids, r1.ids) and np.array_equal(r0.sig, r1.sig))


@pytest.mark.parametrize("seed", [11, 12])
def test_adjoint_matches_finite_differences(orc, seed):
    """Every float input, masks included, against central differences in FP64.

    The scene is perturbed in FP64 (the oracle reads its arrays as given), and
    perturbations whose +-h evaluation flips a discrete decision are skipped."""
    scene, cam, dimg = _fd_scene(seed)
    scene64 = synth.Scene(**{k: (v.astype(np.float64) if v.dtype == np.float32 else v)
                             for k, v in scene.arrays().items()})
    _, res = _loss(orc, scene64, cam, dimg)
    resg = orc.render_forward(scene64, cam, need_grad=True)
    grads = orc.render_backward(resg, scene64, cam, dimg)
    rng = np.random.default_rng(seed)
    checked = 0
    for name in orc.PARAM_NAMES:
        arr = getattr(scene64, name)
        flat = arr.reshape(-1)
        g = grads[name].reshape(-1)
        cand = np.nonzero(g != 0)[0]
        if len(cand) == 0:
            continue
        picks = rng.choice(cand, size=min(6, len(cand)), replace=False)
        for i in picks:
            x0 = flat[i]
            h = 1e-6 * max(1.0, abs(x0))
            flat[i] = x0 + h
            lp, rp = _loss(orc, scene64, cam, dimg)
            flat[i] = x0 - h
            lm, rm = _loss(orc, scene64, cam, dimg)
            flat[i] = x0
            if not (_same_decisions(res, rp) and _same_decisions(res, rm)):
                continue
            fd = (lp - lm) / (2 * h)
            assert fd == pytest.approx(g[i], rel=2e-5, abs=1e-7 * (1 + abs(g).max())), (name, i)
            checked += 1
    assert checked >= 40


def test_adjoint_zero_on_clamped_branches(orc):
    """At the 0.99 clamp the opacity gets no gradient; a colour channel clamped at 0
    passes none back to c0."""
    cam = synth.make_camera(16, 16, 150.0)
    # sigma ~ 110 px: o' G > 0.99 on every pixel of the 16x16 image
    g = one_gaussian_scene((0, 0, 4.0), (3.0,) * 3, opac=0.9995, c0=(-0.3, 0.5, 0.2))
    g64 = synth.Scene(**{k: (v.astype(np.float64) if v.dtype == np.float32 else v)
                         for k, v in g.arrays().items()})
    dimg = np.ones((3, 16, 16))
    r = orc.render_forward(g64, cam, need_grad=True)
    gr = orc.render_backward(r, g64, cam, dimg)
    assert r.T_final.max() == pytest.approx(0.01, rel=1e-12)
    assert gr["opac"][0] == 0.0 and gr["gmask"][0] == 0.0
    assert gr["c0"][0, 0] == 0.0 and gr["c0"][1, 0] > 0


# ---------------------------------------------------------------------------
# Importance score (App. A.2): I_i = sum over rays of alpha_i T_i
# ---------------------------------------------------------------------------

def test_importance_sums_to_coverage(orc):
    """Sum_i I_i = sum over pixels of (1 - T_final): the blend weights of a pixel
    add up to its coverage."""
    rng = np.random.default_rng(31)
    scene = synth.make_scene(rng, 600, lobes=synth.LOBE_MIX, means="cube", masks="uniform")
    cam = synth.make_camera(80, 64, 90.0)
    res = orc.render_forward(scene, cam)
    assert res.importance.sum() == pytest.approx((1 - res.T_final).sum(), rel=1e-12)
    assert (res.importance >= 0).all()
    assert (res.importance[~res.dec.visible] == 0).all()


def test_importance_single_gaussian_closed_form(orc):
    """One Gaussian: I = sum over its pixels of alpha (T = 1 in front of it)."""
    cam = synth.make_camera(48, 48, 150.0)
    g = one_gaussian_scene((0.05, 0.02, 4.0), (0.07,) * 3, opac=0.6)
    res = orc.render_forward(g, cam)
    assert res.importance[0] == pytest.approx((1 - res.T_final).sum(), rel=1e-12)
    # brute force over pixels from the image itself: colour 1 in every channel
    g.c0[:] = 1.0
    res1 = orc.render_forward(g, cam)
    assert res.importance[0] == pytest.approx(res1.img[0].sum(), rel=1e-12)
