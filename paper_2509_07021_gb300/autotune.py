"""Autotuner for the blend kernels' shape (pixels per thread, persistent or
one block per tile) and shared-memory batch size.

Times each candidate on the caller's own scene and cameras with the library's
stage events, picks the fastest forward and backward shape independently, and
caches the choice per (GPU, image sizes, entries) in a JSON file
($SGSPLAT_TUNE_CACHE, default ~/.cache/sgsplat/tune.json).
"""
from __future__ import annotations

import json
import os

import torch

from . import render, sgsplat

CANDIDATES = (1, 2, 4, 8)
FWD_BATCHES = (32, 64, 128)
BWD_BATCHES = (32, 64)


def _cache_path():
    return os.environ.get("SGSPLAT_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "sgsplat", "tune.json"))


def _key(ds, cams):
    name = torch.cuda.get_device_name()
    sizes = ",".join(f"{c.width}x{c.height}" for c in cams)
    # entries rounded to 2 significant digits: nearby scene sizes share a choice
    m = ds.n * len(cams)
    mag = 10 ** max(0, len(str(m)) - 2)
    return f"{name}|{sizes}|{(m // mag) * mag}|{ds.dtype_geom}{ds.dtype_lobe}{ds.dtype_sharp}"


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(data):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def search(measure, candidates=CANDIDATES, persistent=(0, 1)):
    """The search both tuners run. measure(**tuning) sets a tuning, runs the
    workload and returns {"blend_fwd": ms, "blend_bwd": ms}. Every shape
    (pixels per thread x persistent) first, the forward and the backward picked
    independently; then the batch sizes at those shapes. Installs the choice
    and returns it with the timings."""
    timings = {}
    for p, q in [(p, q) for q in persistent for p in candidates]:
        timings[(p, q)] = measure(fwd_pixels_per_thread=p, bwd_pixels_per_thread=p, fwd_persistent=q,
                                  bwd_persistent=q, fwd_batch=0, bwd_batch=0)
    best_f = min(timings, key=lambda k: timings[k]["blend_fwd"])
    best_b = min(timings, key=lambda k: timings[k]["blend_bwd"])
    batch_ms = {}
    for i in range(max(len(FWD_BATCHES), len(BWD_BATCHES))):
        fb = FWD_BATCHES[min(i, len(FWD_BATCHES) - 1)]
        bb = BWD_BATCHES[min(i, len(BWD_BATCHES) - 1)]
        batch_ms[(fb, bb)] = measure(fwd_pixels_per_thread=best_f[0], bwd_pixels_per_thread=best_b[0],
                                     fwd_persistent=best_f[1], bwd_persistent=best_b[1], fwd_batch=fb,
                                     bwd_batch=bb)
    fwd_batch = min(batch_ms, key=lambda k: batch_ms[k]["blend_fwd"])[0]
    bwd_batch = min(batch_ms, key=lambda k: batch_ms[k]["blend_bwd"])[1]
    sgsplat.sg_set_tuning(best_f[0], best_b[0], best_f[1], best_b[1], fwd_batch=fwd_batch, bwd_batch=bwd_batch)
    return {"fwd_pixels_per_thread": best_f[0], "bwd_pixels_per_thread": best_b[0],
            "fwd_persistent": best_f[1], "bwd_persistent": best_b[1],
            "fwd_batch": fwd_batch, "bwd_batch": bwd_batch,
            "ms": {f"p{k[0]}{'_persistent' if k[1] else ''}": v for k, v in timings.items()},
            "batch_ms": {f"fwd{k[0]}_bwd{k[1]}": v for k, v in batch_ms.items()}}


def stage_measure(run, reps):
    """A measure() for search: run() is one forward + backward of the workload;
    timed with the library's stage events over `reps` runs after a warm-up."""
    def measure(**tuning):
        sgsplat.sg_set_tuning(**tuning)
        run()                                          # warm-up for this choice
        torch.cuda.synchronize()
        sgsplat.sg_profile_enable(sgsplat.SG_PROFILE_EVENTS)
        sgsplat.sg_profile_read(reset=True)
        for _ in range(reps):
            run()
        torch.cuda.synchronize()
        st = sgsplat.sg_profile_read(reset=True)["stages"]
        sgsplat.sg_profile_enable(0)
        # every forward builds the tile order (tile_ranges) whatever the shapes, so
        # the blend stages alone tell the shapes apart
        return {"blend_fwd": st["blend_fwd"]["ms"] / reps, "blend_bwd": st["blend_bwd"]["ms"] / reps}
    return measure


def tune(ds, cams, d_img, reps=3, use_cache=True, candidates=CANDIDATES, persistent=(0, 1)):
    """Picks and sets the fastest blend shape (pixels per thread, one block per
    tile or persistent) for the forward and the backward independently on
    this workload. Returns the choice and the timings (ms)."""
    key = _key(ds, cams)
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        c = cache[key]
        sgsplat.sg_set_tuning(c["fwd_pixels_per_thread"], c["bwd_pixels_per_thread"],
                              c.get("fwd_persistent", 0), c.get("bwd_persistent", 0),
                              fwd_batch=c.get("fwd_batch", 0), bwd_batch=c.get("bwd_batch", 0))
        return dict(c, cached=True)
    grads = render.alloc_grads(ds)
    prev = sgsplat.sg_get_tuning()

    def run():
        out = render.render_forward(ds, cams)
        render.render_backward(ds, cams, out, d_img, grads)

    res = search(stage_measure(run, reps), candidates, persistent)
    res["previous"] = prev
    if use_cache:
        cache[key] = res
        _store(cache)
    return dict(res, cached=False)
