"""Property tests of the oracle over random tiny scenes (hypothesis draws the
scene's seed, size, lobe count, image size with ragged tiles, background and
camera pose). Every property follows from the blend sum of Sec. 3.1 and the
tiling rules, independently of how the oracle computes them."""
import numpy as np
import pytest

import oracle as orc
from paper_2509_07021_gb300 import synth

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

SCENES = st.fixed_dictionaries({
    "seed": st.integers(0, 2 ** 32 - 1),
    "n": st.integers(1, 48),
    "lobes": st.sampled_from([0, 1, 4, synth.LOBE_MIX]),
    "w": st.integers(8, 52),
    "h": st.integers(8, 52),
    "bg": st.tuples(*[st.floats(0.0, 1.0)] * 3),
    "eye": st.tuples(st.floats(-0.4, 0.4), st.floats(-0.4, 0.4), st.floats(-0.5, 0.5)),
})


def _draw(d):
    rng = np.random.default_rng(d["seed"])
    scene = synth.make_scene(rng, d["n"], lobes=d["lobes"], means="cube", cube_side=1.2, masks="uniform")
    vm = synth.look_at(d["eye"], (0.0, 0.0, 4.0))
    cam = synth.make_camera(d["w"], d["h"], 1.2 * max(d["w"], d["h"]), bg=d["bg"], viewmat=vm)
    return scene, cam


def _tile_of_pixel(cam):
    ty, tx = np.meshgrid(np.arange(cam.height) // 16, np.arange(cam.width) // 16, indexing="ij")
    return ty * cam.tiles_x + tx


@settings(max_examples=30, deadline=None)
@given(SCENES)
def test_tiled_walk_equals_brute_force(d):
    """The tiled, sorted walk gives exactly the image and transmittance of a
    per-pixel walk over every Gaussian in (depth, index) order gated by its
    3-sigma rectangle."""
    scene, cam = _draw(d)
    res = orc.render_forward(scene, cam)
    img, T, last = orc.brute_force(scene, cam, gate=True)
    np.testing.assert_array_equal(res.img, img)
    np.testing.assert_array_equal(res.T_final, T)
    np.testing.assert_array_equal(res.last, last)


@settings(max_examples=30, deadline=None)
@given(SCENES)
def test_blend_invariants(d):
    """T_final in [1e-4, 1]; the image is at least the background's share;
    the per-Gaussian weights alpha T summed over Gaussians and pixels equal the
    covered amount sum (1 - T_final); every pixel's last contributor lies in its
    tile's list."""
    scene, cam = _draw(d)
    res = orc.render_forward(scene, cam)
    assert (res.T_final >= 1e-4).all() and (res.T_final <= 1.0).all()
    bg = np.asarray(cam.bg, np.float64)
    assert (res.img >= res.T_final[None] * bg[:, None, None] - 1e-12).all()
    np.testing.assert_allclose(res.importance.sum(), (1.0 - res.T_final).sum(), rtol=1e-12, atol=1e-12)
    lens = res.ranges[:, 1] - res.ranges[:, 0]
    assert (res.last <= lens[_tile_of_pixel(cam)]).all()


@settings(max_examples=30, deadline=None)
@given(SCENES)
def test_tile_lists_are_sorted_subsets_of_the_rectangles(d):
    """Each tile's list holds exactly the distinct visible Gaussians whose
    rectangle contains the tile, in ascending (depth bits, index) order."""
    scene, cam = _draw(d)
    dec = orc.decisions_fp32(scene, cam)
    keys, ids, ranges = orc.tile_lists(dec, cam)
    assert len(keys) == len(ids) == int(ranges[:, 1].max(initial=0))
    np.testing.assert_array_equal(np.bincount(ids, minlength=scene.n), dec.touched)
    for t in range(cam.n_tiles):
        a, b = ranges[t]
        g = ids[a:b]
        if len(g) == 0:
            continue
        assert len(np.unique(g)) == len(g)
        assert dec.visible[g].all()
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        r = dec.rect[g]
        assert ((r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])).all()
        order = np.lexsort((g, dec.depth_bits[g]))
        np.testing.assert_array_equal(order, np.arange(len(g)))
        np.testing.assert_array_equal(keys[a:b] >> np.uint64(32), np.full(len(g), t, np.uint64))
