"""CPU oracle of the post-processing procedure (Sec. 3.3.3, Eq. 11-13).
TEST INFRASTRUCTURE ONLY.

Keep decisions are the same binary32 comparisons the library makes
(m_g o is one rounded product); the colour compensation is FP64.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def lobe_mean_factor(s):
    """Mean over the sphere of e^{s (mu.v - 1)}: (1 - e^{-2s}) / (2s), 1 at s = 0 (Eq. 12)."""
    s = np.asarray(s, np.float64)
    out = np.ones_like(s)
    nz = s != 0
    out[nz] = -np.expm1(-2.0 * s[nz]) / (2.0 * s[nz])
    return out


def postprocess(scene, tau_o, tau_s):
    """Returns (kept Gaussian ids, kept lobe ids, new lobe_off, new c0 [3][N'] FP64)."""
    op = scene.gmask.astype(F32) * scene.opac.astype(F32)
    keep_g = op >= F32(tau_o)
    off = scene.lobe_off.astype(np.int64)
    counts = np.diff(off)
    owner = np.repeat(np.arange(scene.n), counts)
    keep_l = keep_g[owner] & (scene.sharp.astype(F32) >= F32(tau_s))
    removed = keep_g[owner] & ~keep_l
    comp = np.zeros((3, scene.n))
    f = scene.lmask.astype(np.float64) * lobe_mean_factor(scene.sharp)
    for d in range(3):
        np.add.at(comp[d], owner[removed], scene.amp[d].astype(np.float64)[removed] * f[removed])
    gid = np.nonzero(keep_g)[0]
    lid = np.nonzero(keep_l)[0]
    new_counts = np.bincount(owner[keep_l], minlength=scene.n)[gid]
    new_off = np.concatenate([[0], np.cumsum(new_counts)]).astype(np.int32)
    c0 = scene.c0.astype(np.float64)[:, gid] + comp[:, gid]
    return gid, lid, new_off, c0
