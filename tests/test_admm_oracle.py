"""Pins of the ADMM-step oracle (Alg. 1, Eq. 7-10)."""
import itertools
import math

import numpy as np
import pytest

from oracle import admm


def test_magnitude_prox_is_the_euclidean_projection():
    """prox_h of the indicator of {||x||_0 <= kappa} (Eq. 6-7) is the nearest
    point of that set: brute force over every support of size kappa."""
    rng = np.random.default_rng(0)
    for n, kappa in ((7, 3), (6, 1), (5, 5), (6, 0)):
        z = rng.normal(0, 1, n)
        best, best_d = None, np.inf
        for S in itertools.combinations(range(n), kappa):
            x = np.zeros(n)
            x[list(S)] = z[list(S)]
            d = np.sum((z - x) ** 2)
            if d < best_d:
                best, best_d = x, d
        got, keep = admm.prox_topk(z, np.abs(z), kappa)
        np.testing.assert_array_equal(got, best)
        assert keep.sum() == kappa


def test_ties_keep_lower_index_and_nan_last():
    z = np.array([1.0, 2.0, 2.0, 5.0, np.nan, 2.0])
    score = np.array([1.0, 2.0, 2.0, 5.0, np.nan, 2.0])
    _, keep = admm.prox_topk(z, score, 3)
    np.testing.assert_array_equal(keep, [False, True, True, True, False, False])
    _, keep = admm.prox_topk(z, score, 6)
    assert keep.all()


def test_dynamic_range_is_max_minus_min_of_the_lobe():
    """Eq. 10 against a dense sampling of mu.v in [-1, 1] (either sign of s)."""
    rng = np.random.default_rng(1)
    t = np.linspace(-1.0, 1.0, 200001)
    for s in (0.3, 2.0, 17.0, -0.7):
        a = rng.normal(0, 1, 3)
        G = np.linalg.norm(a) * np.exp(s * (t - 1.0))
        D = admm.dynamic_range(np.array([s]), a[:, None])[0]
        assert D == pytest.approx(G.max() - G.min(), rel=1e-9)


def test_opacity_step_dual_update_and_sparsity():
    rng = np.random.default_rng(2)
    o = rng.random(50).astype(np.float32)
    lam = rng.normal(0, 0.1, 50).astype(np.float32)
    imp = rng.random(50).astype(np.float32)
    ot, lam2, keep = admm.opacity_step(o, lam, 12, importance=imp)
    assert np.count_nonzero(ot) <= 12 and keep.sum() == 12
    # the kept entries are the 12 most important
    assert set(np.nonzero(keep)[0]) == set(np.argsort(-imp, kind="stable")[:12])
    np.testing.assert_array_equal(ot[keep], (o + lam)[keep])
    # lambda^{k+1} = lambda^k + (o - o~)
    np.testing.assert_allclose(lam2, lam + (o - ot), rtol=0, atol=1e-7)


def test_penalty_grad_is_gradient_of_quadratic():
    rng = np.random.default_rng(3)
    x, xt, lam, g = (rng.normal(0, 1, 9).astype(np.float64) for _ in range(4))
    delta = 5e-4

    def pen(xv):
        return 0.5 * delta * np.sum((xv - xt + lam) ** 2)
    h = 1e-6
    fd = np.array([(pen(x + h * e) - pen(x - h * e)) / (2 * h) for e in np.eye(9)])
    # starting from a zero gradient: no cancellation against g in binary32
    got = admm.penalty_grad(np.zeros(9), x, xt, lam, delta).astype(np.float64)
    np.testing.assert_allclose(got, fd, rtol=1e-5, atol=1e-12)
    # and it adds to a gradient that is already there
    added = admm.penalty_grad(g, x, xt, lam, delta).astype(np.float64)
    np.testing.assert_allclose(added, g.astype(np.float32) + got, rtol=0, atol=2e-7)
