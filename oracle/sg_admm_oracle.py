"""CPU oracle of the ADMM steps of the memory-constrained optimisation (Alg. 1,
Sec. 3.3.2, Eq. 7-10, App. A.2). TEST INFRASTRUCTURE ONLY.

Binary32 where the library computes in binary32 and the result is compared
bit for bit (sums z = x + lambda, the dual update, the penalty term); the
dynamic range D is FP64 (the test allows the kappa-th place to differ only
between scores within rounding of each other).
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def prox_topk(z, score, kappa):
    """Eq. 7-9: keep the kappa entries of z with the largest score (equal
    scores: lower index first; NaN scores last), zero the rest."""
    z = np.asarray(z)
    n = z.shape[0]
    score = np.asarray(score, np.float64)
    key = np.where(np.isnan(score), np.inf, -score)
    order = np.lexsort((np.arange(n), key))
    keep = np.zeros(n, bool)
    keep[order[:max(0, min(int(kappa), n))]] = True
    return np.where(keep, z, z.dtype.type(0)), keep


def opacity_step(o, lam, kappa, importance=None):
    """Proximal step on z = o + lambda (importance-based selection when
    importance is given, magnitude-based otherwise), then the dual update
    lambda + (o - o~). Returns (o~, new lambda, kept mask)."""
    o = np.asarray(o, F32)
    lam = np.asarray(lam, F32)
    z = o + lam
    score = np.abs(z) if importance is None else np.asarray(importance, F32)
    ot, keep = prox_topk(z, score, kappa)
    return ot.astype(F32), (lam + (o - ot)).astype(F32), keep


def dynamic_range(z, amp):
    """Eq. 10: D = |max_v G - min_v G| = |a| |1 - exp(-2 z)| (|a| the RGB norm)."""
    a = np.linalg.norm(np.asarray(amp, np.float64), axis=0)
    return a * np.abs(1.0 - np.exp(-2.0 * np.asarray(z, np.float64)))


def sharpness_step(s, lam, amp, kappa):
    s = np.asarray(s, F32)
    lam = np.asarray(lam, F32)
    z = s + lam
    D = dynamic_range(z, amp)
    st, keep = prox_topk(z, D, kappa)
    return st.astype(F32), (lam + (s - st)).astype(F32), keep, D


def penalty_grad(grad, x, x_tilde, lam, delta):
    """Gradient of delta/2 ||x - x~ + lambda||^2 added to grad (Alg. 1 gradient step)."""
    y = (np.asarray(x, F32) - np.asarray(x_tilde, F32)) + np.asarray(lam, F32)
    return (np.asarray(grad, F32) + F32(delta) * y).astype(F32)
