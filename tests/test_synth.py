"""The seeded input generators follow the stated recipe: lobe mix,
parameter distributions, exact-zero mask fractions, packed means and camera
placement of the five workloads (checked at reduced sizes where the recipe is
per Gaussian)."""
import numpy as np
import pytest

from paper_2509_07021_gb300 import synth


@pytest.fixture(scope="module")
def big():
    return synth.make_scene(np.random.default_rng(1), 200_000, lobes=synth.LOBE_MIX, means="clusters",
                            masks="uniform")


def test_lobe_mix_and_csr(big):
    counts = np.diff(big.lobe_off.astype(np.int64))
    assert big.lobe_off[0] == 0 and big.lobe_off[-1] == big.n_lobes
    for k, p in synth.LOBE_MIX.items():
        assert abs((counts == k).mean() - p) < 0.006, k
    assert abs(counts.mean() - 1.65) < 0.02


def test_parameter_distributions(big):
    ls = np.log(big.scales.astype(np.float64))
    assert abs(ls.mean() + 3.5) < 0.01 and abs(ls.std() - 0.5) < 0.01
    np.testing.assert_allclose(np.linalg.norm(big.quats, axis=0), 1.0, atol=1e-6)
    assert abs(big.quats.mean()) < 0.01
    logit = np.log(big.opac / (1 - big.opac))
    assert abs(logit.mean()) < 0.01 and abs(logit.std() - 1.0) < 0.01
    assert big.c0.min() >= 0 and big.c0.max() <= 1 and abs(big.c0.mean() - 0.5) < 0.01
    np.testing.assert_allclose(np.linalg.norm(big.axis, axis=0), 1.0, atol=1e-6)
    assert np.abs(big.axis.mean(axis=1)).max() < 0.01
    lsh = np.log(big.sharp.astype(np.float64))
    assert lsh.min() >= 0 and lsh.max() <= np.log(50.0) + 1e-6
    assert abs(lsh.mean() - np.log(50.0) / 2) < 0.01
    assert abs(big.amp.std() - 0.3) < 0.005 and abs(big.amp.mean()) < 0.005
    for m in (big.gmask, big.lmask):
        assert m.min() >= 0 and m.max() <= 1 and abs(m.mean() - 0.5) < 0.01


def test_clusters_spread_like_the_recipe(big):
    # 32 cluster centres in a cube of side 10, per-axis std up to 1.5
    assert np.abs(big.means).max() < 5 + 6 * 1.5
    assert 2.0 < big.means.std(axis=1).min() < 4.5


def test_stress_masks_and_packed_means():
    s = synth.make_scene(np.random.default_rng(2), 100_000, lobes=4, means="packed", packed_frac=0.7,
                         masks="uniform", gauss_zero_frac=0.6, lobe_zero_frac=0.5)
    gz = s.gmask == 0
    assert abs(gz.mean() - 0.6) < 0.01
    owner = np.repeat(np.arange(s.n), 4)
    alive = ~gz[owner]
    assert abs((s.lmask[alive] == 0).mean() - 0.5) < 0.01
    r = np.linalg.norm(s.means, axis=0)
    assert abs((r <= 1.5).mean() - (0.7 + 0.3 * (4 / 3 * np.pi * 1.5 ** 3) / 1000)) < 0.01


def test_cameras_of_the_workloads():
    # the 1080p workloads: camera centre (0, 0, -8), looking at the origin
    cam = synth.make_camera(1920, 1080, 1500.0, viewmat=synth.look_at((0.0, 0.0, -8.0), (0.0, 0.0, 0.0)))
    V = cam.viewmat.astype(np.float64)
    np.testing.assert_allclose(-V[:, :3].T @ V[:, 3], [0, 0, -8], atol=1e-6)
    np.testing.assert_allclose(V[:, :3] @ V[:, :3].T, np.eye(3), atol=1e-6)
    np.testing.assert_allclose(V[:, :3] @ np.array([0, 0, 0.0]) + V[:, 3], [0, 0, 8], atol=1e-6)
    # the batched workload: 4 ring cameras per scene, mixed resolutions, same horizontal FOV
    _, cams, _ = synth.config2(sizes=(10, 20))
    assert len(cams) == 2 and all(len(c) == 4 for c in cams)
    for per in cams:
        assert [(c.width, c.height) for c in per] == list(synth.CONFIG2_RES)
        for i, c in enumerate(per):
            assert c.fx == pytest.approx(c.width * 1500.0 / 1920.0)
            V = c.viewmat.astype(np.float64)
            centre = -V[:, :3].T @ V[:, 3]
            assert np.linalg.norm(centre) == pytest.approx(8.0, abs=1e-5)
            th = np.deg2rad(90.0 * i)
            np.testing.assert_allclose(centre, [8 * np.sin(th), 0, -8 * np.cos(th)], atol=1e-5)
    # the stress workload: 16 ring cameras at radius 8, 1600x1066, fx 1250
    ring = synth.ring_cameras(16, 8.0, 1600, 1066, 1250.0)
    centres = np.stack([-c.viewmat[:, :3].T.astype(np.float64) @ c.viewmat[:, 3] for c in ring])
    np.testing.assert_allclose(np.linalg.norm(centres, axis=1), 8.0, atol=1e-5)
    assert len({(round(x, 3), round(z, 3)) for x, _, z in centres}) == 16


def test_seeds_are_reproducible():
    a, _ = synth.config0()
    b, _ = synth.config0()
    for k, v in a.arrays().items():
        np.testing.assert_array_equal(v, getattr(b, k))
