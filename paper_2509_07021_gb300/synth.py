"""Seeded synthetic scenes and cameras.

This module only draws inputs; it holds none of the rasterizer's arithmetic, so
the CUDA path and the CPU oracle can both take their inputs from it.

Scene layout (planar structure of arrays, float32 unless stated):
  means  [3][N]   Gaussian centres (world)
  scales [3][N]   per-axis standard deviations (already activated, > 0)
  quats  [4][N]   rotation quaternion (w, x, y, z), not normalised
  opac   [N]      opacity o in (0, 1)
  gmask  [N]      per-Gaussian soft-pruning mask m_g
  c0     [3][N]   diffuse colour (Sec. 3.2, Eq. 2)
  lobe_off [N+1]  int32 CSR offsets of each Gaussian's SG lobes
  axis   [3][L]   lobe axis mu (Eq. 1), drawn unit length
  sharp  [L]      lobe sharpness s (Eq. 1)
  amp    [3][L]   lobe RGB amplitude a (Eq. 1)
  lmask  [L]      per-lobe soft-pruning mask m_l

The distributions follow the workloads the paper trains on (0.4-2.7 M
Gaussians per scene, Table 13; 0-3 lobes after pruning, Fig. 5) scaled to the
five benchmark workloads built by config0() .. config4() below.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20250907

LOBE_MIX = {0: 0.20, 1: 0.30, 2: 0.25, 3: 0.15, 4: 0.10}


@dataclass
class Camera:
    """Pinhole camera, OpenCV convention (x right, y down, z forward)."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    viewmat: np.ndarray          # (3, 4) float32 world->camera [R | t], row-major
    near: float = 0.2
    bg: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))

    @property
    def tiles_x(self) -> int:
        return (self.width + 15) // 16

    @property
    def tiles_y(self) -> int:
        return (self.height + 15) // 16

    @property
    def n_tiles(self) -> int:
        return self.tiles_x * self.tiles_y

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


@dataclass
class Scene:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opac: np.ndarray
    gmask: np.ndarray
    c0: np.ndarray
    lobe_off: np.ndarray
    axis: np.ndarray
    sharp: np.ndarray
    amp: np.ndarray
    lmask: np.ndarray
    sh: np.ndarray | None = None   # [3][16][N] SH3 coefficients (SH colour model only)

    FLOAT_FIELDS = ("means", "scales", "quats", "opac", "gmask", "c0",
                    "axis", "sharp", "amp", "lmask")

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    @property
    def n_lobes(self) -> int:
        return int(self.sharp.shape[0])

    def arrays(self) -> dict:
        out = {k: getattr(self, k) for k in self.FLOAT_FIELDS + ("lobe_off",)}
        if self.sh is not None:
            out["sh"] = self.sh
        return out

    def copy(self) -> "Scene":
        return Scene(**{k: np.array(v, copy=True) for k, v in self.arrays().items()})

    def param_bytes(self) -> int:
        return sum(int(v.nbytes) for v in self.arrays().values())


def look_at(eye, target, down=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera [R|t] for a camera at `eye` looking at `target` (OpenCV axes)."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    d = np.asarray(down, np.float64)
    y = d - np.dot(d, z) * z
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    rot = np.stack([x, y, z])
    t = -rot @ eye
    return np.concatenate([rot, t[:, None]], axis=1).astype(np.float32)


def make_camera(width, height, fx, fy=None, cx=None, cy=None, viewmat=None,
                near=0.2, bg=(0.0, 0.0, 0.0)) -> Camera:
    fy = fx if fy is None else fy
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    if viewmat is None:
        viewmat = np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32)
    return Camera(int(width), int(height), float(fx), float(fy), float(cx), float(cy),
                  np.asarray(viewmat, np.float32), float(near), np.asarray(bg, np.float32))


def _unit(rng, n, dim):
    v = rng.standard_normal((dim, n))
    return v / np.linalg.norm(v, axis=0, keepdims=True)


def _lobe_counts(rng, n, lobes):
    if isinstance(lobes, int):
        return np.full(n, lobes, np.int64)
    ks = np.array(sorted(lobes), np.int64)
    p = np.array([lobes[k] for k in ks], np.float64)
    return rng.choice(ks, size=n, p=p / p.sum())


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def make_scene(rng, n, *, lobes=LOBE_MIX, means="cube", cube_center=(0.0, 0.0, 4.0),
               cube_side=1.0, n_clusters=32, scene_extent=10.0, masks="ones",
               gauss_zero_frac=0.0, lobe_zero_frac=0.0, packed_frac=0.0,
               packed_radius=1.5) -> Scene:
    """Draw one seeded scene of `n` Gaussians.

    means: "cube"     uniform in an axis-aligned cube (side `cube_side`)
           "clusters" mixture of `n_clusters` anisotropic 3D Gaussian clusters,
                      centres uniform in a cube of side `scene_extent`, per-cluster
                      random rotation and per-axis std U[0.3, 1.5], equal weights
           "packed"   `packed_frac` of the means uniform in a ball of radius
                      `packed_radius` at the origin, the rest uniform in the cube
    masks: "ones" | "uniform" (U(0,1)); then `gauss_zero_frac` of the Gaussians get
           m_g = 0 exactly and `lobe_zero_frac` of the remaining Gaussians' lobes
           get m_l = 0 exactly.
    """
    counts = _lobe_counts(rng, n, lobes)
    lobe_off = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=lobe_off[1:])
    n_l = int(lobe_off[-1])

    if means == "cube":
        c = np.asarray(cube_center, np.float64)[:, None]
        mu = c + (rng.random((3, n)) - 0.5) * cube_side
    elif means == "clusters":
        half = scene_extent / 2.0
        centres = rng.uniform(-half, half, (n_clusters, 3))
        rots = np.stack([_random_rotation(rng) for _ in range(n_clusters)])
        stds = rng.uniform(0.3, 1.5, (n_clusters, 3))
        which = rng.integers(0, n_clusters, n)
        eps = rng.standard_normal((n, 3)) * stds[which]
        mu = (centres[which] + np.einsum("nij,nj->ni", rots[which], eps)).T
    elif means == "packed":
        half = scene_extent / 2.0
        n_in = int(round(packed_frac * n))
        d = _unit(rng, n_in, 3)
        r = packed_radius * rng.random(n_in) ** (1.0 / 3.0)
        inner = d * r
        outer = rng.uniform(-half, half, (3, n - n_in))
        mu = np.concatenate([inner, outer], axis=1)
        mu = mu[:, rng.permutation(n)]
    else:
        raise ValueError(means)

    scales = np.exp(rng.normal(-3.5, 0.5, (3, n)))
    quats = rng.standard_normal((4, n))
    quats /= np.linalg.norm(quats, axis=0, keepdims=True)
    opac = _sigmoid(rng.standard_normal(n))
    c0 = rng.random((3, n))
    axis = _unit(rng, n_l, 3)
    sharp = np.exp(rng.uniform(np.log(1.0), np.log(50.0), n_l))
    amp = rng.normal(0.0, 0.3, (3, n_l))

    if masks == "ones":
        gmask = np.ones(n)
        lmask = np.ones(n_l)
    elif masks == "uniform":
        gmask = rng.uniform(0.0, 1.0, n)
        lmask = rng.uniform(0.0, 1.0, n_l)
    else:
        raise ValueError(masks)
    if gauss_zero_frac > 0:
        gz = rng.random(n) < gauss_zero_frac
        gmask[gz] = 0.0
        owner = np.repeat(np.arange(n), counts)
        alive_lobe = ~gz[owner]
        lz = alive_lobe & (rng.random(n_l) < lobe_zero_frac)
        lmask[lz] = 0.0

    f = np.float32
    return Scene(means=mu.astype(f), scales=scales.astype(f), quats=quats.astype(f),
                 opac=opac.astype(f), gmask=gmask.astype(f), c0=c0.astype(f),
                 lobe_off=lobe_off.astype(np.int32), axis=axis.astype(f),
                 sharp=sharp.astype(f), amp=amp.astype(f), lmask=lmask.astype(f))


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def ring_cameras(n, radius, width, height, fx, start_deg=0.0):
    """`n` cameras on a horizontal ring of `radius` around the origin, looking in."""
    cams = []
    for i in range(n):
        th = np.deg2rad(start_deg + 360.0 * i / n)
        eye = (radius * np.sin(th), 0.0, -radius * np.cos(th))
        cams.append(make_camera(width, height, fx, viewmat=look_at(eye, (0.0, 0.0, 0.0))))
    return cams


def upstream_grad(rng, cam: Camera, std=0.01) -> np.ndarray:
    """dL/dimg ~ N(0, std) per pixel and channel, shape [3][H][W] float32."""
    return rng.normal(0.0, std, (3, cam.height, cam.width)).astype(np.float32)


def rng_for(config: int, salt: int = 0):
    return np.random.default_rng(SEED_BASE + config + 1000 * salt)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def config0():
    """1,000 Gaussians, 3 lobes each, 128x128 camera at the origin looking +z."""
    rng = rng_for(0)
    scene = make_scene(rng, 1000, lobes=3, means="cube")
    cam = make_camera(128, 128, 150.0)
    return scene, [cam]


def config_single_1080p(n, config, masks="uniform"):
    """`n` Gaussians in 32 clusters, one 1920x1080 camera at distance 8 (fx=1500)."""
    rng = rng_for(config)
    scene = make_scene(rng, n, lobes=LOBE_MIX, means="clusters", masks=masks)
    cam = make_camera(1920, 1080, 1500.0, viewmat=look_at((0.0, 0.0, -8.0), (0.0, 0.0, 0.0)))
    return scene, [cam], rng


def config1():
    return config_single_1080p(500_000, 1)


def config3():
    return config_single_1080p(1_000_000, 3)


CONFIG2_SIZES = (50_000, 120_000, 300_000, 600_000, 900_000, 1_200_000, 1_500_000, 2_000_000)
CONFIG2_RES = ((800, 800), (1280, 720), (1600, 1066), (1920, 1080))


def config2(sizes=CONFIG2_SIZES):
    """Uneven scenes, each seen by 4 ring cameras at mixed resolutions."""
    rng = rng_for(2)
    scenes, cams = [], []
    for n in sizes:
        scenes.append(make_scene(rng, n, lobes=LOBE_MIX, means="clusters", masks="uniform"))
        per = []
        for i, (w, h) in enumerate(CONFIG2_RES):
            th = np.deg2rad(90.0 * i)
            eye = (8.0 * np.sin(th), 0.0, -8.0 * np.cos(th))
            per.append(make_camera(w, h, w * 1500.0 / 1920.0,
                                   viewmat=look_at(eye, (0.0, 0.0, 0.0))))
        cams.append(per)
    return scenes, cams, rng


def config4(n=6_000_000, n_cams=16):
    """Stress form: packed cluster, 4 lobes, 60% / 50% exact-zero masks, 16 ring cameras."""
    rng = rng_for(4)
    scene = make_scene(rng, n, lobes=4, means="packed", packed_frac=0.7, masks="uniform",
                       gauss_zero_frac=0.6, lobe_zero_frac=0.5)
    cams = ring_cameras(n_cams, 8.0, 1600, 1066, 1250.0)
    return scene, cams, rng


STORAGE_FAMILIES = {
    # storage form -> {field: dtype name}; fields not listed stay binary32
    "f32": {},
    "f16": {k: "float16" for k in ("means", "scales", "quats", "opac", "axis", "amp", "sharp")},
    "f16_bf16s": dict({k: "float16" for k in ("means", "scales", "quats", "opac", "axis", "amp")},
                      sharp="bfloat16"),
}


def round_to_storage(scene: Scene, storage: str) -> Scene:
    """The binary32 values a scene holds after a round trip through `storage`
    (what the kernels read back from half-precision arrays)."""
    import torch
    out = scene.copy()
    for k, dt in STORAGE_FAMILIES[storage].items():
        t = torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32))
        setattr(out, k, t.to(getattr(torch, dt)).float().numpy())
    return out


def with_sh3_colour(scene: Scene, rng, dc_std=1.0, band_std=0.2) -> Scene:
    """The same geometry with a degree-3 SH colour instead of SG lobes:
    coefficients [3][16][N] (DC ~ N(0, dc_std), higher bands ~ N(0, band_std)),
    no lobes, c0 unused (zeros)."""
    n = scene.n
    sh = rng.normal(0.0, band_std, (3, 16, n))
    sh[:, 0, :] = rng.normal(0.0, dc_std, (3, n))
    f = np.float32
    out = scene.copy()
    out.sh = sh.astype(f)
    out.c0 = np.zeros((3, n), f)
    out.lobe_off = np.zeros(n + 1, np.int32)
    out.axis = np.zeros((3, 0), f)
    out.sharp = np.zeros(0, f)
    out.amp = np.zeros((3, 0), f)
    out.lmask = np.zeros(0, f)
    return out
