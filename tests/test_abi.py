"""C ABI checks that need no GPU: the library loads, exports every function
include/sgsplat.h declares, sizes workspaces on the host, and rejects bad
arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

from paper_2509_07021_gb300 import sgsplat, synth
from paper_2509_07021_gb300.sgsplat import DeviceScene

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2509_07021_gb300 import build
    if not os.path.exists(build.library_path()):
        build.build()
    return sgsplat.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert {"sg_render_forward", "sg_render_backward", "sg_workspace_query"} <= set(names)
    for n in names:
        assert hasattr(L, n), n
    assert set(sgsplat.EXPORTS) <= set(names)


def test_version(L):
    assert sgsplat.sg_version() == 1


def _cpu_scene(n=100, lobes=2):
    """A DeviceScene whose tensors live on the CPU: only its sizes are used by the
    host-only calls below (pointers are never dereferenced there)."""
    s = synth.make_scene(np.random.default_rng(0), n, lobes=lobes)
    return DeviceScene.from_host(s, device="cpu")


def test_workspace_query_sizes(L):
    ds = _cpu_scene(1000, 3)
    cams = [synth.make_camera(128, 96, 150.0), synth.make_camera(64, 64, 80.0)]
    q0 = sgsplat.sg_workspace_query(ds, cams, 0)
    q1 = sgsplat.sg_workspace_query(ds, cams, 100_000)
    assert q0["n_entries"] == 2000
    assert q0["n_tiles"] == 8 * 6 + 4 * 4
    assert q0["n_pixels"] == 128 * 96 + 64 * 64
    assert q0["ws_fixed_bytes"] == q0["ws_bytes"] == q1["ws_fixed_bytes"]
    # 64 tiles: the tile sort counts, so 10 bytes of pair buffers per pair (the
    # duplicate's 16-bit keys and entries, the sorted entries) plus its count
    # matrix; the depth sort's buffers (16 bytes per entry) live in the pair
    # buffers' memory (regions aligned to 256 bytes)
    diff = q1["ws_bytes"] - q1["ws_fixed_bytes"]
    assert 10 * 100_000 - 16 * 2000 - 1024 <= diff <= 12 * 100_000 + 4096
    assert q1["ws_per_pair_bytes"] >= 10
    assert q1["bwd_ws_bytes"] >= 9 * 4 * 2000
    lay = sgsplat.sg_workspace_layout(ds, cams, q1["ws_bytes"])
    assert lay["total_bytes"] == q1["ws_bytes"]
    # the counting sort keeps no sorted tile ids
    assert lay["pair_tile"] == 2**64 - 1
    offs = sorted(v for k, v in lay.items() if k not in ("total_bytes", "pair_tile"))
    assert all(o % 256 == 0 for o in offs)
    assert len(set(offs)) == len(offs)


def test_tile_sort_path_follows_the_tile_count(L):
    """Up to 12288 tiles in all the tile sort counts: 16-bit duplicate keys, the
    sorted entries only (pair_tile absent), a count matrix of at most 608 rows
    of the padded tile count in the look-back flags' region. Above it the radix
    passes keep sorted tile ids in two 16-byte-per-pair regions."""
    ds = _cpu_scene(1000, 2)
    cap = 2_000_000
    # 1920x1080: 120 x 68 = 8160 tiles (counting); two such views: 16320 (radix)
    one = [synth.make_camera(1920, 1080, 1500.0)]
    two = one * 2
    q1 = sgsplat.sg_workspace_query(ds, one, cap)
    q2 = sgsplat.sg_workspace_query(ds, two, cap)
    assert q1["n_tiles"] == 8160 and q2["n_tiles"] == 16320
    l1 = sgsplat.sg_workspace_layout(ds, one, q1["ws_bytes"])
    l2 = sgsplat.sg_workspace_layout(ds, two, q2["ws_bytes"])
    assert l1["pair_tile"] == 2**64 - 1
    assert l2["pair_tile"] != 2**64 - 1 and l2["pair_tile"] % 256 == 0
    assert q1["pair_capacity"] == cap and q2["pair_capacity"] == cap
    # per pair of capacity: 10 bytes of pairs + the matrix share (4 B x 8160
    # tiles per 8192 pairs) against 16 bytes of pairs + the radix flags
    assert q1["ws_per_pair_bytes"] == 10 + 4 and q2["ws_per_pair_bytes"] == 17
    f1 = q1["ws_bytes"] - q1["ws_fixed_bytes"]
    f2 = q2["ws_bytes"] - q2["ws_fixed_bytes"]
    chunks = min(608, -(-cap // 8192))
    assert f1 <= 10 * cap + 4 * 8160 * chunks + 4096
    assert f2 >= 16 * cap - 16 * 2000
    # at the counting limit (12288 tiles: 2048 x 1536) and one tile row past it
    at = [synth.make_camera(2048, 1536, 1500.0)]
    past = [synth.make_camera(2048, 1552, 1500.0)]
    assert sgsplat.sg_workspace_query(ds, at, 0)["n_tiles"] == 12288
    assert sgsplat.sg_workspace_query(ds, past, 0)["n_tiles"] == 12416
    la = sgsplat.sg_workspace_layout(ds, at, sgsplat.sg_workspace_query(ds, at, cap)["ws_bytes"])
    lp = sgsplat.sg_workspace_layout(ds, past, sgsplat.sg_workspace_query(ds, past, cap)["ws_bytes"])
    assert la["pair_tile"] == 2**64 - 1
    assert lp["pair_tile"] != 2**64 - 1


def _status(L, fn, *args):
    return fn(*args)


def test_invalid_arguments_rejected_on_host(L):
    ds = _cpu_scene(10, 1)
    s = ds.struct()
    cams = sgsplat.camera_array([synth.make_camera(32, 32, 40.0)])
    out = sgsplat.sg_sizes()
    P = ctypes.c_void_p
    # no cameras
    assert L.sg_workspace_query(ctypes.byref(s), None, 1, 0, ctypes.byref(out)) == sgsplat.SG_ERR_INVALID_ARG
    # n_views out of range
    assert L.sg_workspace_query(ctypes.byref(s), cams, 0, 0, ctypes.byref(out)) == sgsplat.SG_ERR_INVALID_ARG
    assert L.sg_workspace_query(ctypes.byref(s), cams, 129, 0, ctypes.byref(out)) == sgsplat.SG_ERR_INVALID_ARG
    # bad dtype
    s2 = ds.struct()
    s2.dtype_geom = 7
    assert L.sg_workspace_query(ctypes.byref(s2), cams, 1, 0, ctypes.byref(out)) == sgsplat.SG_ERR_INVALID_ARG
    assert "dtype" in sgsplat.sg_last_error()
    # negative size
    s3 = ds.struct()
    s3.n = -1
    assert L.sg_workspace_query(ctypes.byref(s3), cams, 1, 0, ctypes.byref(out)) == sgsplat.SG_ERR_INVALID_ARG
    # zero-sized image and non-finite intrinsics
    bad = sgsplat.camera_array([synth.make_camera(32, 32, 40.0)])
    bad[0].width = 0
    assert L.sg_workspace_query(ctypes.byref(s), bad, 1, 0, ctypes.byref(out)) == sgsplat.SG_ERR_INVALID_ARG
    bad = sgsplat.camera_array([synth.make_camera(32, 32, 40.0)])
    bad[0].fx = float("nan")
    assert L.sg_workspace_query(ctypes.byref(s), bad, 1, 0, ctypes.byref(out)) == sgsplat.SG_ERR_INVALID_ARG
    # forward: NULL outputs, NULL / misaligned workspace are refused before any device work
    st = L.sg_render_forward(ctypes.byref(s), cams, 1, P(256), 1 << 20, None, None, None,
                             ctypes.byref(out), None)
    assert st == sgsplat.SG_ERR_INVALID_ARG
    st = L.sg_render_forward(ctypes.byref(s), cams, 1, P(8), 1 << 20, P(256), P(256), P(256),
                             ctypes.byref(out), None)
    assert st == sgsplat.SG_ERR_INVALID_ARG
    # misaligned scene array
    s4 = ds.struct()
    s4.means = 4
    st = L.sg_render_forward(ctypes.byref(s4), cams, 1, P(256), 1 << 20, P(256), P(256), P(256),
                             ctypes.byref(out), None)
    assert st == sgsplat.SG_ERR_INVALID_ARG and "aligned" in sgsplat.sg_last_error()
    # backward: missing gradient struct
    st = L.sg_render_backward(ctypes.byref(s), cams, 1, P(256), 1 << 20, P(256), P(256), P(256),
                              P(256), 1 << 20, None, None)
    assert st == sgsplat.SG_ERR_INVALID_ARG


def test_batched_arguments_rejected_on_host(L):
    a, b = _cpu_scene(10, 1), _cpu_scene(20, 2)
    cams = [synth.make_camera(32, 32, 40.0), synth.make_camera(48, 16, 40.0)]
    q = sgsplat.sg_batched_workspace_query([a, b], cams, [0, 1], 1000)
    assert q["n_entries"] == 30 and q["n_tiles"] == 4 + 3
    # a view of a scene the call does not hold
    with pytest.raises(sgsplat.SGError) as e:
        sgsplat.sg_batched_workspace_query([a, b], cams, [0, 2], 0)
    assert e.value.status == sgsplat.SG_ERR_INVALID_ARG and "scene index" in str(e.value)
    # the scenes of one call share their storage types
    h = DeviceScene.from_host(synth.make_scene(np.random.default_rng(1), 10, lobes=1), device="cpu",
                              storage="f16")
    with pytest.raises(sgsplat.SGError) as e:
        sgsplat.sg_batched_workspace_query([a, h], cams, [0, 1], 0)
    assert e.value.status == sgsplat.SG_ERR_INVALID_ARG and "share" in str(e.value)


def test_noalloc_backward_rejected_on_host(L):
    """The no-alloc backward refuses a missing gradient struct, a misaligned
    workspace and a call whose scratch exceeds its static array, before it
    touches a device."""
    ds = _cpu_scene(10, 1)
    cams = sgsplat.camera_array([synth.make_camera(32, 32, 40.0)])
    P = ctypes.c_void_p
    g = sgsplat.grads_struct({})
    s = ds.struct()
    st = L.sg_render_backward_noalloc(ctypes.byref(s), cams, 1, P(256), 1 << 20, P(256), P(256), P(256),
                                      None, None)
    assert st == sgsplat.SG_ERR_INVALID_ARG
    st = L.sg_render_backward_noalloc(ctypes.byref(s), cams, 1, P(8), 1 << 20, P(256), P(256), P(256),
                                      ctypes.byref(g), None)
    assert st == sgsplat.SG_ERR_INVALID_ARG and "aligned" in sgsplat.sg_last_error()
    big = ds.struct()
    big.n = sgsplat.SG_NOALLOC_SCRATCH_BYTES // 36 + 1000   # sizes only: never dereferenced
    st = L.sg_render_backward_noalloc(ctypes.byref(big), cams, 1, P(256), 1 << 20, P(256), P(256),
                                      P(256), ctypes.byref(g), None)
    assert st == sgsplat.SG_ERR_WORKSPACE and "static scratch" in sgsplat.sg_last_error()


def test_workspace_too_small_for_fixed_part(L):
    ds = _cpu_scene(10, 1)
    cams = [synth.make_camera(32, 32, 40.0)]
    with pytest.raises(sgsplat.SGError) as e:
        sgsplat.sg_workspace_layout(ds, cams, 64)
    assert e.value.status == sgsplat.SG_ERR_WORKSPACE


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2509_07021_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), f
                assert "sg_blend_oracle" not in src and "liborc" not in src, f
