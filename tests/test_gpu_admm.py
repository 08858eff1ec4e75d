"""ADMM steps on the GPU (Alg. 1) vs the oracle: selections and updates bit
exact where the scores are inputs or exact binary32 sums; the dynamic-range
selection may differ only between scores within rounding of the kappa-th."""
import numpy as np
import pytest
import torch

from oracle import admm
from paper_2509_07021_gb300 import sgsplat

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("n,kappa", [(1000, 137), (70000, 25000), (5, 0), (9, 9), (4097, 4096)])
@pytest.mark.parametrize("importance", [True, False])
def test_opacity_step(n, kappa, importance):
    rng = np.random.default_rng(n + kappa)
    o = rng.random(n).astype(np.float32)
    lam = rng.normal(0, 0.2, n).astype(np.float32)
    imp = rng.random(n).astype(np.float32) if importance else None
    if importance:
        imp[::7] = imp[0]          # ties: lower index first
    ot_ref, lam_ref, keep = admm.opacity_step(o, lam, kappa, imp)
    lam_d, ot_d = _t(lam), torch.full((n,), float("nan"), device="cuda")
    sgsplat.sg_admm_opacity_step(_t(o), lam_d, ot_d, kappa, importance=None if imp is None else _t(imp))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ot_d.cpu().numpy(), ot_ref)
    np.testing.assert_array_equal(lam_d.cpu().numpy(), lam_ref)


@pytest.mark.parametrize("L,kappa", [(3000, 1000), (100000, 33333)])
def test_sharpness_step(L, kappa):
    rng = np.random.default_rng(L)
    s = np.exp(rng.uniform(0, np.log(50), L)).astype(np.float32)
    s[::11] = rng.normal(0, 0.5, s[::11].size)      # some near zero or negative
    lam = rng.normal(0, 0.3, L).astype(np.float32)
    amp = rng.normal(0, 0.3, (3, L)).astype(np.float32)
    st_ref, lam_ref, keep_ref, D = admm.sharpness_step(s, lam, amp, kappa)
    lam_d, st_d = _t(lam), torch.zeros(L, device="cuda")
    sgsplat.sg_admm_sharpness_step(_t(s), _t(amp), lam_d, st_d, kappa)
    torch.cuda.synchronize()
    st = st_d.cpu().numpy()
    keep = st != 0
    z = (s + lam).astype(np.float32)
    keep |= (z == 0) & keep_ref      # z exactly 0 kept looks like dropped
    thr = np.sort(D)[::-1][kappa - 1]
    sure_in = D > thr * (1 + 1e-5)
    sure_out = D < thr * (1 - 1e-5)
    assert keep[sure_in].all() and not keep[sure_out].any()
    assert keep.sum() == kappa
    np.testing.assert_array_equal(st[keep], z[keep])
    np.testing.assert_array_equal(lam_d.cpu().numpy(), (lam + (s - st)).astype(np.float32))


def test_penalty_grad_bit_exact():
    rng = np.random.default_rng(9)
    x, xt, lam, g = (rng.normal(0, 1, 5000).astype(np.float32) for _ in range(4))
    gd = _t(g)
    sgsplat.sg_admm_penalty_grad(_t(x), _t(xt), _t(lam), 5e-4, gd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(gd.cpu().numpy(), admm.penalty_grad(g, x, xt, lam, 5e-4))


@pytest.mark.parametrize("kappa", [1, 4000, 12345, 20000])
def test_opacity_step_ties_across_blocks(kappa):
    """The kappa-th score lies in a run of equal scores that spans many blocks
    of the selection's final pass: the kept ties are the lowest indices."""
    rng = np.random.default_rng(kappa)
    n = 30000
    o = rng.random(n).astype(np.float32)
    lam = rng.normal(0, 0.2, n).astype(np.float32)
    imp = np.where(rng.random(n) < 0.7, np.float32(0.5), rng.random(n).astype(np.float32)).astype(np.float32)
    ot_ref, lam_ref, keep = admm.opacity_step(o, lam, kappa, imp)
    lam_d, ot_d = _t(lam), torch.full((n,), float("nan"), device="cuda")
    sgsplat.sg_admm_opacity_step(_t(o), lam_d, ot_d, kappa, importance=_t(imp))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ot_d.cpu().numpy(), ot_ref)
    np.testing.assert_array_equal(lam_d.cpu().numpy(), lam_ref)
