"""Pins of the post-processing oracle (Sec. 3.3.3, Eq. 11-13)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import post
from paper_2509_07021_gb300 import synth


def _sphere_rule(nu=300, nphi=96):
    u, wu = np.polynomial.legendre.leggauss(nu)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    U, PHI = np.meshgrid(u, phi, indexing="ij")
    st = np.sqrt(1 - U ** 2)
    v = np.stack([st * np.cos(PHI), st * np.sin(PHI), U], -1).reshape(-1, 3)
    w = (wu[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    return v, w


def _colour(scene, g, v):
    """Eq. 2 colour (before the clamp) of Gaussian g of `scene` in directions v."""
    lo, hi = scene.lobe_off[g], scene.lobe_off[g + 1]
    n = v.shape[0]
    t = lambda a: torch.tensor(np.asarray(a, np.float64))
    c0 = t(np.tile(scene.c0[:, g], (n, 1)))
    k = np.arange(lo, hi)
    off = np.concatenate([[0], np.cumsum(np.full(n, hi - lo))])
    rep = lambda a: t(np.tile(a[..., k].T if a.ndim == 2 else a[k], (n, 1) if a.ndim == 2 else n)
                      .reshape(-1, 3) if a.ndim == 2 else np.tile(a[k], n))
    return oracle.sg_color(c0, off, rep(scene.axis), rep(scene.sharp), rep(scene.amp),
                           rep(scene.lmask), t(v)).numpy()


def test_compensation_preserves_the_mean_colour_over_the_sphere():
    """Eq. 11: the compensation is the constant closest (in L2 over S^2) to the
    removed lobes, i.e. their mean -- so the colour's mean is unchanged."""
    rng = np.random.default_rng(0)
    scene = synth.make_scene(rng, 12, lobes=4, masks="uniform")
    scene.sharp[:] = rng.choice([0.0, 0.05, 0.5, 0.99, 1.0, 3.0, 20.0], scene.n_lobes).astype(np.float32)
    scene.gmask[:] = 1.0
    gid, lid, off, c0 = post.postprocess(scene, 0.0, 1.0)
    assert len(gid) == scene.n and len(lid) == int((scene.sharp >= 1.0).sum())
    out = scene.copy()
    out.c0 = c0.astype(np.float64)
    out.lobe_off = off
    for k in ("axis", "amp"):
        setattr(out, k, getattr(scene, k)[:, lid])
    for k in ("sharp", "lmask"):
        setattr(out, k, getattr(scene, k)[lid])
    v, w = _sphere_rule()
    for g in range(scene.n):
        before = (_colour(scene, g, v) * w[:, None]).sum(0) / (4 * np.pi)
        after = (_colour(out, g, v) * w[:, None]).sum(0) / (4 * np.pi)
        np.testing.assert_allclose(after, before, rtol=1e-9, atol=1e-12)


def test_lobe_mean_factor_limits():
    assert post.lobe_mean_factor(np.array([0.0]))[0] == 1.0
    s = np.array([1e-8, -1e-8, 2.0, -0.5])
    np.testing.assert_allclose(post.lobe_mean_factor(s),
                               (1 - np.exp(-2 * s)) / (2 * s), rtol=1e-7)


def test_opacity_threshold_and_order():
    rng = np.random.default_rng(1)
    scene = synth.make_scene(rng, 200, lobes=synth.LOBE_MIX, masks="uniform")
    gid, lid, off, c0 = post.postprocess(scene, 0.3, 1e9)   # drop every lobe
    eff = scene.gmask.astype(np.float32) * scene.opac.astype(np.float32)
    np.testing.assert_array_equal(gid, np.nonzero(eff >= np.float32(0.3))[0])
    assert len(lid) == 0 and (off == 0).all()
