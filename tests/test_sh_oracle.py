"""Pins of the oracle's degree-3 SH colour (the 3DGS baseline colour model).

The basis is checked against what fixes it independently of the oracle's
construction: orthonormality on the sphere by exact quadrature, the complex
spherical harmonics of scipy (same Condon-Shortley phase), the textbook degree-1
functions, the addition theorem per band, and a render-level reduction
to the SG model with no lobes. The adjoint w.r.t. the SH coefficients and the
means (through the view direction) is pinned by FP64 central differences.
"""
import math

import numpy as np
import pytest
import torch

from paper_2509_07021_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_sh_basis_orthonormal(orc):
    """Gauss-Legendre in z (8 nodes) x 16 uniform azimuths integrates every
    product of two degree-3 harmonics exactly: the Gram matrix is the identity."""
    zn, zw = np.polynomial.legendre.leggauss(8)
    phi = np.arange(16) * (2 * math.pi / 16)
    Z, PHI = np.meshgrid(zn, phi, indexing="ij")
    st = np.sqrt(1 - Z ** 2)
    v = np.stack([st * np.cos(PHI), st * np.sin(PHI), Z], -1).reshape(-1, 3)
    w = (zw[:, None] * np.full(16, 2 * math.pi / 16)[None, :]).reshape(-1)
    Y = orc.sh.basis(torch.from_numpy(v)).numpy()
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_matches_scipy_complex_harmonics(orc):
    """Real form of scipy's complex Y_l^m (Condon-Shortley phase included):
    m > 0: sqrt2 Re Y_l^m, m < 0: sqrt2 Im Y_l^|m|, m = 0: Y_l^0."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(3)
    v = _unit(rng, 64)
    theta = np.arccos(np.clip(v[:, 2], -1, 1))     # polar
    phi = np.arctan2(v[:, 1], v[:, 0])             # azimuth
    Y = orc.sh.basis(torch.from_numpy(v)).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            if hasattr(sp, "sph_harm_y"):
                yc = sp.sph_harm_y(l, abs(m), theta, phi)
            else:
                yc = sp.sph_harm(abs(m), l, phi, theta)
            ref = yc.real if m == 0 else math.sqrt(2) * (yc.real if m > 0 else yc.imag)
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-12, err_msg=f"l={l} m={m}")


def test_sh_degree0_and_degree1_textbook(orc):
    """Y_0 = 1 / (2 sqrt(pi)); the degree-1 band is sqrt(3 / (4 pi)) (-y, z, -x)."""
    rng = np.random.default_rng(4)
    v = _unit(rng, 20)
    Y = orc.sh.basis(torch.from_numpy(v)).numpy()
    np.testing.assert_allclose(Y[:, 0], 0.5 / math.sqrt(math.pi), rtol=1e-14)
    k = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[:, 1:4], k * np.stack([-v[:, 1], v[:, 2], -v[:, 0]], 1), rtol=1e-13)


def test_sh_band_energy_rotation_invariant(orc):
    """sum_m Y_l^m(v)^2 = (2l + 1) / (4 pi) for every direction (addition theorem)."""
    rng = np.random.default_rng(5)
    v = _unit(rng, 50)
    Y = orc.sh.basis(torch.from_numpy(v)).numpy()
    for l in range(4):
        band = Y[:, l * l:(l + 1) * (l + 1)]
        np.testing.assert_allclose((band ** 2).sum(1), (2 * l + 1) / (4 * math.pi), rtol=1e-12)


def _sg_scene_no_lobes(seed, n=12):
    rng = np.random.default_rng(seed)
    s = synth.make_scene(rng, n, lobes=0, means="cube", masks="uniform")
    s.scales *= 3.0
    return s, rng


def test_sh_dc_only_equals_sg_without_lobes(orc):
    """A DC-only SH colour 0.5 + f0 / (2 sqrt(pi)) renders the same image as the
    SG model with c0 = that constant and no lobes."""
    sg, rng = _sg_scene_no_lobes(21)
    cam = synth.make_camera(40, 36, 45.0, bg=(0.3, 0.1, 0.6))
    shs = synth.with_sh3_colour(sg, rng, band_std=0.0)
    c = 0.5 + shs.sh[:, 0, :].astype(np.float64) * (0.5 / math.sqrt(math.pi))
    sg64 = synth.Scene(**{k: v for k, v in sg.arrays().items()})
    sg64.c0 = c
    a = orc.render_forward(sg64, cam).img
    b = orc.render_forward(shs, cam).img
    np.testing.assert_allclose(b, a, atol=1e-13)


def test_sh_adjoint_matches_finite_differences(orc):
    """SH coefficients and means (the view direction moves with the mean)
    against FP64 central differences."""
    sg, rng = _sg_scene_no_lobes(22, n=14)
    scene = synth.with_sh3_colour(sg, rng)
    scene64 = synth.Scene(**{k: (v.astype(np.float64) if v.dtype == np.float32 else v)
                             for k, v in scene.arrays().items()})
    cam = synth.make_camera(40, 36, 45.0, bg=(0.3, 0.1, 0.6))
    dimg = rng.normal(0, 1, (3, cam.height, cam.width))
    r = orc.render_forward(scene64, cam, need_grad=True)
    grads = orc.render_backward(r, scene64, cam, dimg)
    assert grads["sh"].shape == scene.sh.shape

    def loss():
        res = orc.render_forward(scene64, cam)
        return float((res.img * dimg).sum()), res

    checked = 0
    for name in ("sh", "means", "opac"):
        flat = getattr(scene64, name).reshape(-1)
        g = grads[name].reshape(-1)
        cand = np.nonzero(g != 0)[0]
        picks = rng.choice(cand, size=min(10, len(cand)), replace=False)
        for i in picks:
            x0 = flat[i]
            h = 1e-6 * max(1.0, abs(x0))
            flat[i] = x0 + h
            lp, rp = loss()
            flat[i] = x0 - h
            lm, rm = loss()
            flat[i] = x0
            if not (np.array_equal(rp.ids, r.ids) and np.array_equal(rm.ids, r.ids)
                    and np.array_equal(rp.sig, r.sig) and np.array_equal(rm.sig, r.sig)):
                continue
            fd = (lp - lm) / (2 * h)
            assert fd == pytest.approx(g[i], rel=2e-5, abs=1e-7 * (1 + abs(g).max())), (name, i)
            checked += 1
    assert checked >= 20


def test_sh_adjoint_zero_on_clamped_channel(orc):
    """A channel whose colour is clamped at 0 for every view direction passes no
    gradient to its 16 coefficients; the other channels do get one."""
    sg, rng = _sg_scene_no_lobes(23, n=6)
    scene = synth.with_sh3_colour(sg, rng)
    scene.sh[0, :, :] = 0.0
    scene.sh[0, 0, :] = -20.0        # red = 0.5 - 20 / (2 sqrt(pi)) < 0 everywhere
    cam = synth.make_camera(40, 36, 45.0)
    dimg = np.ones((3, cam.height, cam.width))
    r = orc.render_forward(scene, cam, need_grad=True)
    g = orc.render_backward(r, scene, cam, dimg)
    vis = r.dec.visible
    assert vis.any()
    assert np.all(g["sh"][0] == 0.0)
    assert np.abs(g["sh"][1][:, vis]).max() > 0
