#!/usr/bin/env python
"""Benchmark: forward + backward of the SG-splatting rasterizer.

One step = one forward (preprocessSG, depth sort, duplicateWithKeys, tile sort,
ranges, blend) and one backward (blend adjoint, preprocess adjoint) of one
1920x1080 view of a synthetic 1M-Gaussian scene with 0-4 SG lobes per Gaussian
(mix 20/30/25/15/10 %), soft masks U(0,1), and an upstream image gradient
N(0, 0.01). Inputs are resident in HBM; L2 is flushed between timed steps.

Prints ONE JSON line. `--impl reference` times the FP64 CPU oracle instead
(the only place besides the cpu_baseline leg where bench.py runs it).
Multi-GPU (torchrun): independent replicas, one per rank, no collective on the
data path (weak scaling); rank 0 prints the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/view & Mpixel/s (1080p, 1M Gaussians, ≤4 SG); batched vs plain"
UNIT = "Mpixel/s"
L2_FLUSH_BYTES = 512 << 20

# Algorithmic FP32 work per evaluated (pixel, Gaussian) pair, FMA = 2 flops:
# forward 23 (quadratic form, exponent, alpha tests, transmittance and colour
# update), backward 69 (about 14 for power and alpha, 46 for the adjoint, 9 for
# the warp reduction amortised over the pairs).
FLOPS_PER_EVAL = {"blend_fwd": 23.0, "blend_bwd": 69.0}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each
# stage's kernel at this workload, from one ncu capture, together with the
# digest of the CUDA sources it was taken on: reported as roofline.traffic only
# while the sources are unchanged (any kernel change makes it null until the
# next capture).
RECORDED_TRAFFIC = {
    "sources": "080aff9b363c692f75aa9f2580e8ba2acb293f3bbe3a982abbdad2eae7efd4a0",
    "bytes": {"blend_bwd": 120819456, "blend_fwd": 50263552},
}


def kernel_source_digest(root=None):
    """sha256 over the CUDA sources (any kernel change invalidates recorded counters)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(root or ROOT, "paper_2509_07021_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def recorded_traffic(stage, table=None, root=None):
    """DRAM bytes per launch of a stage's kernel from the recorded capture, or
    None when the sources changed since (or the stage was not captured)."""
    table = RECORDED_TRAFFIC if table is None else table
    if not table.get("sources") or table["sources"] != kernel_source_digest(root):
        return None
    v = table.get("bytes", {}).get(stage)
    return None if v is None else float(v)


# GB300 FP32 (non-tensor) peak: 152 SMs x 128 lanes x 2 flops x 2.07 GHz
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.07
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1e3


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "f16", "f16_bf16s"], default="f32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP16-storage, batched and stress forms")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default blend shapes")
    ap.add_argument("--shape", default="",
                    help="fixed blend shape fwd_ppt,bwd_ppt,fwd_persistent,bwd_persistent (no autotune)")
    ap.add_argument("--cpu-tiles", type=int, default=48,
                    help="tiles of the frame the CPU oracle blends per sample")
    return ap.parse_args()


def workload():
    from paper_2509_07021_gb300 import synth
    scene, cams, rng = synth.config3()
    d_img = synth.upstream_grad(np.random.default_rng(synth.SEED_BASE + 33), cams[0])
    return scene, cams, d_img


def workload_config(args, cams, extra=None):
    c = cams[0]
    cfg = {"workload": f"1M Gaussians, {c.width}x{c.height}, lobes 0-4 (mix 20/30/25/15/10%), "
                       f"masks U(0,1), {args.storage} storage, fwd+bwd, 1 view/step",
           "n_gaussians": 1_000_000, "width": c.width, "height": c.height, "views_per_step": 1,
           "storage": args.storage, "l2": "flushed between timed steps (512 MiB write)",
           "parallelism": f"replicas x{args.gpus}"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# distributed helpers (replicas only)
# ---------------------------------------------------------------------------

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples (20 ms) with timestamps; summarises those that fall in
    the timed window (widened by `pad` seconds when the window is shorter than
    a few samples)."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self, interval_ms=50, ready_timeout=10.0):
        """Starts nvidia-smi and returns once its first sample is on file, so
        that its start-up never overlaps a timed region."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(int(interval_ms))],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < ready_timeout and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.05)
        except Exception:
            self.proc = None

    def stop(self, t0, t1, pad=0.25):
        import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if t0 <= r[0] <= t1]
        window = "timed region"
        if len(inside) < 3:
            inside = [r for r in rows if t0 - pad <= r[0] <= t1 + pad]
            window = f"timed region +-{pad}s"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = sorted({self.NAMES[i] for r in inside for i in range(4) if r[3][i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside), "reasons": reasons,
                "samples": len(inside), "window": window}


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline / --impl reference)
# ---------------------------------------------------------------------------

def oracle_fixed_time(scene, cam):
    """Seconds of the oracle's full-frame part of a step: decisions and the
    tile lists of every tile."""
    import oracle
    t0 = time.perf_counter()
    dec = oracle.decisions_fp32(scene, cam)
    oracle.tile_lists(dec, cam)
    return time.perf_counter() - t0


def oracle_sample(scene, cam, d_img, n_tiles, seed=0, t_fixed=None):
    """One bounded oracle sample of the workload: the full-frame preprocess and
    tile lists, then forward + backward blend on n_tiles random tiles (upstream
    gradient restricted to them). t_fixed: the seconds of the full-frame part
    (oracle_fixed_time), measured here when not given. Returns (seconds of
    the sample, estimated seconds for the whole frame, threads)."""
    import oracle
    if t_fixed is None:
        t_fixed = oracle_fixed_time(scene, cam)
    sel = np.zeros(cam.n_tiles, bool)
    sel[np.random.default_rng(seed).choice(cam.n_tiles, n_tiles, replace=False)] = True
    t1 = time.perf_counter()
    res = oracle.render_forward(scene, cam, tile_sel=sel, need_grad=True)
    m = np.repeat(np.repeat(sel.reshape(cam.tiles_y, cam.tiles_x), 16, 0), 16, 1)
    m = m[:cam.height, :cam.width]
    oracle.render_backward(res, scene, cam, d_img * m[None])
    t_sample = time.perf_counter() - t1
    # the sample holds the full-frame part once; scale the rest (the blend of
    # the sampled tiles) to the whole frame
    t_blend = max(t_sample - t_fixed, 0.0)
    est_full = t_sample - t_blend + t_blend * cam.n_tiles / n_tiles
    return t_sample, est_full, oracle.num_threads()


def cpu_baseline_line(scene, cam, d_img, n_tiles):
    """The oracle on the host cores: all cores (the reported value), then one
    thread on a smaller sample, then the small forward-only workload in full."""
    import oracle
    import torch
    total, est_full, threads = oracle_sample(scene, cam, d_img, n_tiles)
    mpx = cam.width * cam.height / 1e6
    line = {"value": mpx / est_full, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"FP64 oracle: full-frame preprocess + tile sort, forward+backward blend on "
                       f"{n_tiles} of {cam.n_tiles} random tiles ({total:.1f} s wall), blend time "
                       f"scaled to the frame; {threads} OpenMP threads for the blend, numpy/torch "
                       f"for the rest")}
    torch_threads = torch.get_num_threads()
    try:
        oracle.set_num_threads(1)
        torch.set_num_threads(1)
        n1 = max(4, n_tiles // 4)
        total1, est1, _ = oracle_sample(scene, cam, d_img, n1, seed=1)
        line["single_thread"] = {"value": mpx / est1, "unit": UNIT, "cores": 1,
                                 "sample": f"same, {n1} random tiles, one thread ({total1:.1f} s wall)"}
    finally:
        oracle.set_num_threads(threads)
        torch.set_num_threads(torch_threads)
    from paper_2509_07021_gb300 import synth
    s0, c0 = synth.config0()
    t0 = time.perf_counter()
    oracle.render_forward(s0, c0[0])
    dt = time.perf_counter() - t0
    line["small_forward"] = {"ms_per_view": 1e3 * dt, "workload": "1,000 Gaussians x 3 lobes, 128x128, "
                             "forward only, whole frame", "cores": threads}
    s1, c1, _ = synth.config1()
    d1 = synth.upstream_grad(np.random.default_rng(synth.SEED_BASE + 11), c1[0])
    n1 = max(4, n_tiles // 3)
    total_h, est_h, _ = oracle_sample(s1, c1[0], d1, n1, seed=2)
    line["half_million"] = {"value": mpx / est_h, "unit": UNIT, "s_per_view": est_h, "cores": threads,
                            "workload": "500k Gaussians, 1920x1080, lobes 0-4, fwd+bwd",
                            "sample": f"full-frame preprocess + tile sort, blend on {n1} random tiles "
                                      f"scaled to the frame ({total_h:.1f} s wall)"}
    return line


def gpu_errors_vs_oracle(scene, cam, d_img, storages=("f32", "f16_bf16s"), n_tiles=24, seed=5):
    """Image max / mean abs error and per-tensor gradient relative L2 of the GPU
    forms against the FP64 oracle on a sample of tiles: the upstream gradient is
    d_img on those tiles (zero elsewhere and at the oracle's ambiguous pixels),
    and the oracle is fed the original binary32 scene (so the half-storage
    numbers include the storage rounding)."""
    import oracle
    import torch
    from paper_2509_07021_gb300 import render
    from paper_2509_07021_gb300.sgsplat import DeviceScene
    sel = np.zeros(cam.n_tiles, bool)
    sel[np.random.default_rng(seed).choice(cam.n_tiles, n_tiles, replace=False)] = True
    res = oracle.render_forward(scene, cam, tile_sel=sel, need_grad=True)
    m = np.repeat(np.repeat(sel.reshape(cam.tiles_y, cam.tiles_x), 16, 0), 16, 1)
    m = m[:cam.height, :cam.width] & ~res.ambiguous
    dimg = (d_img * m[None]).astype(np.float32)
    g_orc = oracle.render_backward(res, scene, cam, dimg)
    out = {}
    for storage in storages:
        ds = DeviceScene.from_host(scene, storage=storage)
        fwd = render.render_forward(ds, [cam])
        g = render.render_backward(ds, [cam], fwd, torch.from_numpy(dimg)[None].cuda())
        torch.cuda.synchronize()
        img = fwd.img[0].cpu().numpy()
        err = np.abs(img - res.img)[:, m]
        rel = {}
        for k, ref in g_orc.items():
            got = g[k].cpu().numpy().astype(np.float64)
            nr = np.linalg.norm(ref)
            if ref.size and nr > 0:
                rel[k] = float(np.linalg.norm(got - ref) / nr)
        out[storage] = {"img_max_abs": float(err.max()), "img_mean_abs": float(err.mean()),
                        "pixels": int(m.sum()), "grad_rel_l2_max": max(rel.values()), "grad_rel_l2": rel}
        del ds, fwd, g
    return out


def stage_rooflines(stages_ms, counts, evals, hbm_gbs):
    """Achieved fraction of roofline for every stage: algorithmic bytes (HBM
    stages) or flops (blend) per step over the stage's event time per step.
    counts: N Gaussians, L lobes, M entries, V entries with pairs, K pairs, T tiles;
    counting: the tile sort counted (cap: the pair capacity, which sets its chunks)."""
    N, L, M, V, K, T = (counts[k] for k in ("N", "L", "M", "V", "K", "T"))
    by = {
        "preprocess": 64 * N + 32 * L + 69 * M,                 # params in; record, tt, rect, clamp, key, value out
        "depth_sort": 4 * M + 8 * M + 8 * V + 3 * 16 * V,       # histogram, pass 0 (drops), passes 1-3
        "pair_offsets": 12 * V,                                 # sorted id + tt in, offset out
        "duplicate": 64 * V + 8 * K,                            # id, tt, rect, record in; pairs out
        "tile_sort": 4 * K + 2 * 16 * K + 8 * T,                # histogram, two passes, tile ranges
        "tile_ranges": 12 * T,                                  # persistent tile order: ranges in, order out
        "bwd_clear": 36 * M,
        "preprocess_bwd": 64 * N + 32 * L + 41 * M + 60 * N + 32 * L,
    }
    if counts.get("counting"):
        # chunks of the counting tile sort (at most 608, 8192 pairs of capacity each)
        C = min(608, max(1, -(-int(counts["cap"]) // 8192)))
        by["duplicate"] = 64 * V + 6 * K                        # 16-bit tile keys
        # keys read twice, entries read and written; the [C][T] count matrix written,
        # read and rewritten by the scan, read by the placing; tile ranges
        by["tile_sort"] = 4 * K + 8 * K + 16 * C * T + 8 * T
    out = {}
    for k, ms in stages_ms.items():
        if ms <= 0:
            continue
        if k in FLOPS_PER_EVAL:
            ev = evals["forward" if k == "blend_fwd" else "backward"]
            a = ev * FLOPS_PER_EVAL[k] / (ms / 1e3) / 1e12
            out[k] = {"bound": "alu", "achieved": round(a, 2), "unit": "TFLOP/s",
                      "frac": round(a / FP32_PEAK_TFLOPS, 3)}
        elif k in by:
            a = by[k] / (ms / 1e3) / 1e9
            out[k] = {"bound": "hbm", "achieved": round(a, 1), "unit": "GB/s", "frac": round(a / hbm_gbs, 3),
                      "bytes": int(by[k])}
    return out


def step_stats(ms):
    """min / median / mean / max of per-step milliseconds."""
    return {"min": float(min(ms)), "median": float(statistics.median(ms)), "mean": float(statistics.mean(ms)),
            "max": float(max(ms))}


def run_reference(args, world, rank):
    if rank != 0:
        return
    scene, cams, d_img = workload()
    cam = cams[0]
    n_tiles = max(4, args.cpu_tiles // 3)
    t_fixed = oracle_fixed_time(scene, cam)
    for _ in range(args.warmup):
        oracle_sample(scene, cam, d_img, n_tiles, t_fixed=t_fixed)
    ests, totals = [], []
    threads = 1
    for i in range(args.steps):
        total, est, threads = oracle_sample(scene, cam, d_img, n_tiles, seed=i, t_fixed=t_fixed)
        ests.append(est)
        totals.append(total)
    frame_ms = 1e3 * float(np.mean(ests))
    value = cam.width * cam.height / 1e6 / (frame_ms / 1e3)
    wall_ms = 1e3 * float(np.mean(totals))
    sample = (f"each step: full-frame preprocess + tile sort, fwd+bwd blend on {n_tiles} random tiles "
              f"(measured wall {wall_ms / 1e3:.1f} s/step); value = the frame's pixels over the frame "
              f"time estimated by scaling the blend part to all {cam.n_tiles} tiles "
              f"({frame_ms / 1e3:.1f} s/frame)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall_ms,
            "frame_ms_estimate": frame_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, cams),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import torch
    from paper_2509_07021_gb300 import render, sgsplat
    from paper_2509_07021_gb300.sgsplat import DeviceScene

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    sgsplat.lib()   # fails loudly if the extension is missing
    scene, cams, d_img_np = workload()
    cam = cams[0]
    ds = DeviceScene.from_host(scene, device="cuda", storage=args.storage)
    d_img = torch.from_numpy(d_img_np)[None].cuda()
    grads = render.alloc_grads(ds)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step():
        out = render.render_forward(ds, cams)
        render.render_backward(ds, cams, out, d_img, grads)
        return out

    clocks = ClockSampler(local)
    clocks.start()
    tuned = None
    if args.shape:
        f, b, fp, bp = (int(x) for x in args.shape.split(","))
        sgsplat.sg_set_tuning(f, b, fp, bp)
    elif not args.no_autotune:
        from paper_2509_07021_gb300 import autotune
        tuned = autotune.tune(ds, cams, d_img, use_cache=False)
    for _ in range(max(args.warmup, 1)):
        out = step()
    torch.cuda.synchronize()
    n_pairs = out.sizes["n_pairs"]

    # pair evaluations (counting kernels, untimed)
    sgsplat.sg_profile_enable(sgsplat.SG_PROFILE_COUNT)
    sgsplat.sg_profile_read(reset=True)
    step()
    torch.cuda.synchronize()
    evals = sgsplat.sg_profile_read(reset=True)["pair_evals"]
    sgsplat.sg_profile_enable(0)

    # ---- stage breakdown (untimed pass, every stage bracketed by events) ----
    sgsplat.sg_profile_set_stages(0xFFFFFFFF)
    sgsplat.sg_profile_enable(sgsplat.SG_PROFILE_EVENTS)
    sgsplat.sg_profile_read(reset=True)
    n_break = max(3, min(args.steps, 10))
    for i in range(n_break):
        flush.fill_(i & 0xFF)
        step()
    torch.cuda.synchronize()
    fl_stages = {k: v for k, v in sgsplat.sg_profile_read(reset=True)["stages"].items() if v["launches"]}
    dom = max(fl_stages, key=lambda k: fl_stages[k]["ms"])
    tot_stage_ms = max(sum(x["ms"] for x in fl_stages.values()), 1e-9)
    share = {k: round(v["ms"] / tot_stage_ms, 4) for k, v in fl_stages.items()}
    stages_ms = {k: round(v["ms"] / n_break, 4) for k, v in fl_stages.items()}

    # ---- timed region: W fresh warm-up steps right before it (the GPU is not
    # left idle in between), then K steps, each bracketed by CUDA events and
    # synchronised, the L2 flushed before each; only the dominant stage is
    # bracketed inside the step, for its live average launch duration ----
    dom_index = [sgsplat.sg_profile_stage_name(i) for i in range(sgsplat.SG_PROFILE_STAGES)].index(dom)
    sgsplat.sg_profile_set_stages(1 << dom_index)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    def timed_steps():
        for i in range(max(args.warmup, 1)):
            flush.fill_(i & 0xFF)
            step()
        torch.cuda.synchronize()
        sgsplat.sg_profile_read(reset=True)
        barrier(world)
        torch.cuda.synchronize()
        n0 = sgsplat.sg_kernel_launches()
        t0 = time.time()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            starts[i].record()
            step()
            ends[i].record()
            ends[i].synchronize()
        t1 = time.time()
        n1 = sgsplat.sg_kernel_launches()
        barrier(world)
        return [s.elapsed_time(e) for s, e in zip(starts, ends)], t0, t1, n1 - n0

    per_step, wall0, wall1, launches = timed_steps()
    clk = clocks.stop(wall0, wall1)
    prof = sgsplat.sg_profile_read(reset=True)
    # the same K steps again with the clock sampler stopped (does sampling disturb the steps?)
    check_steps, _, _, _ = timed_steps()
    sgsplat.sg_profile_enable(0)
    sgsplat.sg_profile_read(reset=True)
    stats = step_stats(per_step)
    ms_step = max_over_ranks(stats["median"], world)
    px = cam.width * cam.height
    value = world * px / (ms_step / 1e3) / 1e6

    sgsplat.sg_profile_set_stages(0xFFFFFFFF)

    # ---- roofline of the dominant kernel (its events inside the timed region) ----
    stages = prof["stages"]
    avg_ms = stages[dom]["ms"] / max(stages[dom]["launches"], 1)
    if dom in FLOPS_PER_EVAL:
        ev = evals["forward" if dom == "blend_fwd" else "backward"]
        achieved = ev * FLOPS_PER_EVAL[dom] / (avg_ms / 1e3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": recorded_traffic(dom),
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz (FP32 non-tensor)",
                "pair_evals": ev, "flops_per_eval": FLOPS_PER_EVAL[dom], "avg_ms": avg_ms}
    else:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s",
                "frac": None, "traffic": recorded_traffic(dom), "avg_ms": avg_ms}

    # ---- every stage against its roofline (stage times from the breakdown pass) ----
    lay = sgsplat.sg_workspace_layout(ds, cams, out.ws.numel())
    M = out.sizes["n_entries"]
    tt = out.ws[lay["tiles_touched"]:lay["tiles_touched"] + 4 * M].view(torch.int32)
    counts = {"N": scene.n, "L": scene.n_lobes, "M": M, "V": int((tt != 0).sum().item()),
              "K": n_pairs, "T": cam.n_tiles, "cap": out.sizes["pair_capacity"],
              "counting": lay["pair_tile"] == 2**64 - 1}
    hbm_peak = 6800.0
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        pass
    kernel_roofs = stage_rooflines(stages_ms, counts, evals, hbm_peak)

    # ---- end to end through the public API with host buffers ----
    e2e = run_e2e(args, ds, cams, d_img_np, grads, world)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, cams),
            "step_ms": dict(stats, timing="CUDA events per step, synchronised each step; ms_per_step is "
                                          "the median", per_step=[round(x, 4) for x in per_step]),
            "timing_check": {"sampler_off": step_stats(check_steps),
                             "note": "the same K steps again with the nvidia-smi sampler stopped"},
            "workload_stats": {"n_pairs": n_pairs, "tuning": sgsplat.sg_get_tuning(),
                               "autotune_ms": tuned and tuned.get("ms")},
            "roofline": roof, "clocks": clk, "e2e": e2e,
            "gpu_launches": int(launches),
            "stages_ms_per_step": stages_ms,
            "stage_share": share,
            "kernel_rooflines": {"counts": counts, "hbm_peak_gbs": hbm_peak, "stages": kernel_roofs},
            "pair_evals": evals}
    if world == 1 and not args.no_forms:
        forms = run_forms(args, scene, cams, d_img, flush, max(3, args.steps // 2), hbm_peak)
        forms.pop("_images")
        if not args.no_cpu_baseline:
            errs = gpu_errors_vs_oracle(scene, cam, d_img_np)
            forms["plain_f32"]["vs_oracle"] = errs["f32"]
            forms["plain_f16_bf16s"]["vs_oracle"] = errs["f16_bf16s"]
        line["forms"] = forms
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(scene, cam, d_img_np, args.cpu_tiles)
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the other forms of the metric: FP16 storage, batched (config 2), stress (4)
# ---------------------------------------------------------------------------

def _timed(fn, steps, warmup, flush):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for i in range(steps):
        flush.fill_(i & 0xFF)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def next_rows(scene, cams, flush, steps, hbm_gbs):
    """Time and roofline of the rows built after the render path, on the bench
    scene: the importance score fused into the forward (against the plain
    forward), the ADMM steps of Alg. 1 over the N opacities and the L lobes
    (kappa = half of them), and the post-processing (plan + apply). The HBM
    fraction counts each array read and written once (the top-kappa selections
    also sort their scores: that traffic is not counted)."""
    import torch
    from paper_2509_07021_gb300 import render, sgsplat
    from paper_2509_07021_gb300.sgsplat import DeviceScene
    out = {}
    ds = DeviceScene.from_host(scene)
    N, L = ds.n, int(ds.sharp.numel())
    imp = torch.zeros(N, device="cuda")
    ms_plain = _timed(lambda: render.render_forward(ds, cams), steps, 2, flush)
    ms_imp = _timed(lambda: render.render_forward(ds, cams, importance=imp), steps, 2, flush)
    out["importance_forward"] = {"ms": ms_imp, "plain_forward_ms": ms_plain,
                                 "overhead": ms_imp / ms_plain - 1.0,
                                 "nonzero": int((imp > 0).sum().item()), "gaussians": N}

    def hbm(name, ms, nbytes, n, extra=None):
        a = nbytes / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "n": n, "bytes": int(nbytes), "achieved_gbs": round(a, 1),
                     "frac": round(a / hbm_gbs, 3), **(extra or {})}

    g = torch.Generator(device="cuda").manual_seed(7)
    lam_o = torch.randn(N, device="cuda", generator=g) * 0.2
    ot = torch.empty(N, device="cuda")
    ws = sgsplat.sg_admm_opacity_step(ds.opac, lam_o.clone(), ot, N // 2, importance=imp)
    lam_w = lam_o.clone()
    ms = _timed(lambda: sgsplat.sg_admm_opacity_step(ds.opac, lam_w, ot, N // 2, importance=imp, ws=ws),
                steps, 2, flush)
    hbm("admm_opacity_step", ms, 20 * N, N, {"kappa": N // 2, "score": "importance"})
    lam_s = torch.randn(L, device="cuda", generator=g) * 0.3
    st = torch.empty(L, device="cuda")
    ws_s = sgsplat.sg_admm_sharpness_step(ds.sharp, ds.amp, lam_s.clone(), st, L // 2)
    ms = _timed(lambda: sgsplat.sg_admm_sharpness_step(ds.sharp, ds.amp, lam_s, st, L // 2, ws=ws_s),
                steps, 2, flush)
    hbm("admm_sharpness_step", ms, 28 * L, L, {"kappa": L // 2, "score": "dynamic range"})
    grad = torch.zeros(N, device="cuda")
    ms = _timed(lambda: sgsplat.sg_admm_penalty_grad(ds.opac, ot, lam_o, 1e-3, grad), steps, 2, flush)
    hbm("admm_penalty_grad", ms, 20 * N, N)
    ms = _timed(lambda: sgsplat.sg_postprocess(ds, 0.05), steps, 2, flush)
    kept = sgsplat.sg_postprocess(ds, 0.05)
    nb = 64 * N + 32 * L + 64 * kept.n + 32 * int(kept.sharp.numel())
    hbm("postprocess", ms, nb, N, {"tau_opacity": 0.05, "kept_gaussians": kept.n,
                                   "kept_lobes": int(kept.sharp.numel()),
                                   "note": "plan + apply, including the output allocation"})
    del ds, kept
    torch.cuda.empty_cache()
    return out


def render_vram(ds, cams, d_img, grads, static_bytes):
    """Rendering VRAM as the paper measures it (PyTorch allocator peak during a
    render, static parameters included): static parameter bytes + the peak
    the render adds over what was allocated before it (workspace, outputs).
    Returned for a forward only and for forward + backward (gradients and
    upstream gradient buffers are counted as allocated by the caller)."""
    import torch
    from paper_2509_07021_gb300 import render
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    before = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    out = render.render_forward(ds, cams)
    torch.cuda.synchronize()
    fwd_peak = torch.cuda.max_memory_allocated() - before
    render.render_backward(ds, cams, out, d_img, grads)
    torch.cuda.synchronize()
    both = torch.cuda.max_memory_allocated() - before
    grads_bytes = sum(g.numel() * g.element_size() for g in grads.values())
    del out
    return static_bytes + fwd_peak, static_bytes + both + grads_bytes + d_img.numel() * 4


def run_forms(args, scene, cams, d_img, flush, steps, hbm_gbs=6800.0):
    """Timing (and VRAM / error) of the storage and batched forms."""
    import torch
    from paper_2509_07021_gb300 import render, sgsplat, synth
    from paper_2509_07021_gb300.sgsplat import DeviceScene
    forms = {}
    cam = cams[0]
    px = cam.width * cam.height

    # ---- plain FP32 vs FP16/BF16 storage, same scene and view ----
    base = {}
    for storage in ("f32", "f16_bf16s"):
        torch.cuda.empty_cache()
        ds = DeviceScene.from_host(scene, storage=storage)
        grads = render.alloc_grads(ds)
        static = sum(getattr(ds, k).numel() * getattr(ds, k).element_size()
                     for k in DeviceScene.FLOAT_FIELDS + ("lobe_off",))
        fwd_peak, both_peak = render_vram(ds, cams, d_img, grads, static)

        def step():
            out = render.render_forward(ds, cams)
            render.render_backward(ds, cams, out, d_img, grads)
        ms = _timed(step, steps, 2, flush)
        out = render.render_forward(ds, cams)
        torch.cuda.synchronize()
        base[storage] = out.img[0].cpu().numpy()
        forms[f"plain_{storage}"] = {"ms_per_view": ms, "mpixel_s": px / ms / 1e3,
                                     "static_mb": static / 2**20, "render_vram_mb": fwd_peak / 2**20,
                                     "fwd_bwd_vram_mb": both_peak / 2**20}
        del ds, grads, out
    f32, f16 = forms["plain_f32"], forms["plain_f16_bf16s"]
    f16["speedup_vs_plain_f32"] = f32["ms_per_view"] / f16["ms_per_view"]
    f16["render_vram_reduction"] = 1.0 - f16["render_vram_mb"] / f32["render_vram_mb"]
    f16["max_abs_img_diff_vs_f32_gpu"] = float(np.abs(base["f16_bf16s"] - base["f32"]).max())
    forms["_images"] = base   # consumed by the oracle error report, removed before printing

    # ---- the same step through the graph-capturable form: one scene, one view,
    # the same upstream gradient, forward + backward replayed as one CUDA graph ----
    torch.cuda.empty_cache()
    ds = DeviceScene.from_host(scene)
    br = render.BatchedRenderer([ds], cams, [0])
    br.d_img.copy_(d_img.reshape(-1))
    br.capture(None)
    ms = _timed(br.replay, steps, 2, flush)
    n_pairs_g, status_g = br.status()
    forms["graph_f32"] = {"ms_per_view": ms, "mpixel_s": px / ms / 1e3, "n_pairs": n_pairs_g,
                          "status": status_g, "pair_capacity": br.capacity,
                          "speedup_vs_plain_f32": f32["ms_per_view"] / ms}
    del br, ds

    # ---- the 3DGS baseline colour: degree-3 SH (48 floats per Gaussian) on the same geometry ----
    torch.cuda.empty_cache()
    sh_scene = synth.with_sh3_colour(scene, np.random.default_rng(synth.SEED_BASE + 5))
    ds = DeviceScene.from_host(sh_scene)
    del sh_scene
    grads = render.alloc_grads(ds)
    static = sum(getattr(ds, k).numel() * getattr(ds, k).element_size()
                 for k in ("means", "scales", "quats", "opac", "gmask", "sh"))
    fwd_peak, both_peak = render_vram(ds, cams, d_img, grads, static)

    def step_sh():
        out = render.render_forward(ds, cams)
        render.render_backward(ds, cams, out, d_img, grads)
    ms = _timed(step_sh, steps, 2, flush)
    forms["plain_sh3_f32"] = {"ms_per_view": ms, "mpixel_s": px / ms / 1e3, "static_mb": static / 2**20,
                              "render_vram_mb": fwd_peak / 2**20, "fwd_bwd_vram_mb": both_peak / 2**20,
                              "sg_static_reduction": 1.0 - f32["static_mb"] / (static / 2**20)}
    del ds, grads

    # ---- the rows after the render path: importance, ADMM steps, post-processing ----
    torch.cuda.empty_cache()
    forms["next_rows"] = next_rows(scene, cams, flush, steps, hbm_gbs)

    # ---- batched: 8 uneven scenes x 4 cameras, one CUDA graph ----
    for name, gen in (("batched_cfg2", synth.config2), ("stress_cfg4", synth.config4)):
        torch.cuda.empty_cache()
        if name == "batched_cfg2":
            scenes, cams_per, rng = gen()
            all_cams = [c for cs in cams_per for c in cs]
            view_scene = [s for s, cs in enumerate(cams_per) for _ in cs]
        else:
            sc, all_cams, rng = gen()
            scenes = [sc]
            view_scene = [0] * len(all_cams)
        dss = [DeviceScene.from_host(s_) for s_ in scenes]
        del scenes
        br = render.BatchedRenderer(dss, all_cams, view_scene)
        gen_t = torch.Generator(device="cuda").manual_seed(synth.SEED_BASE + 2)
        targets = torch.rand(br.img.shape, device="cuda", generator=gen_t)
        lg = render.l1_loss_grad(br, targets)
        # this batch's own shapes and batch sizes (the plain loop below keeps the
        # single-view workload's)
        main_tuning = sgsplat.sg_get_tuning()
        tuned_b = br.autotune(lg) if not args.no_autotune else None
        batch_tuning = sgsplat.sg_get_tuning()
        br.capture(lg)
        ms_b = _timed(br.replay, max(3, steps // 2), 2, flush)
        n_pairs, status = br.status()
        sgsplat.sg_set_tuning(**main_tuning)
        P = int(br.offsets[-1])
        # the same work through the plain single-view renderer, view by view
        plain_grads = [render.alloc_grads(d) for d in dss]

        def plain_loop():
            for v, c in enumerate(all_cams):
                d = dss[view_scene[v]]
                out = render.render_forward(d, [c])
                o, n = int(br.offsets[v]), br.npix[v]
                tgt = targets[3 * o:3 * (o + n)].view(1, 3, c.height, c.width)
                g = torch.sign(out.img - tgt) / (3 * n)
                render.render_backward(d, [c], out, g, plain_grads[view_scene[v]])
        ms_p = _timed(plain_loop, 2, 1, flush)
        forms[name] = {"views": len(all_cams), "scenes": len(dss),
                       "gaussians": int(sum(d.n for d in dss)), "mpixels": P / 1e6,
                       "n_pairs": n_pairs, "status": status,
                       "ms_per_launch": ms_b, "ms_per_view": ms_b / len(all_cams),
                       "mpixel_s": P / ms_b / 1e3, "plain_loop_ms": ms_p,
                       "speedup_vs_plain_loop": ms_p / ms_b,
                       "tuning": batch_tuning, "plain_loop_tuning": sgsplat.sg_get_tuning(),
                       "autotune_ms": tuned_b and tuned_b.get("ms")}
        del br, dss, plain_grads, targets
        torch.cuda.empty_cache()
    return forms


def run_e2e(args, ds, cams, d_img_np, grads, world):
    """Same metric through the public API with pinned host inputs and outputs:
    every step copies the scene and the upstream gradient host->device and the
    image and all gradients device->host. The value is that of
    render.HostPipeline (steps queued back to back, each step's copies
    overlapped with its neighbours' compute); the serial render.HostStep (one
    step at a time, returning with its results on the host) is reported
    beside it."""
    import torch
    from paper_2509_07021_gb300 import render
    from paper_2509_07021_gb300.sgsplat import DeviceScene

    fields = list(DeviceScene.FLOAT_FIELDS) + ["lobe_off"]
    host_in = {k: getattr(ds, k).cpu().pin_memory() for k in fields}
    host_dimg = torch.from_numpy(d_img_np)[None].pin_memory()
    host_img = torch.empty((1, 3, cams[0].height, cams[0].width), dtype=torch.float32).pin_memory()
    host_grads = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in grads.items()}
    px = cams[0].width * cams[0].height

    step = render.HostStep(ds, cams, host_in, host_dimg, host_img, host_grads)
    for _ in range(max(1, args.warmup)):
        step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    t_serial = max_over_ranks((time.perf_counter() - t0) / args.steps, world)

    pipe = render.HostPipeline(ds, cams)
    h2d, d2h = pipe.bytes_moved(host_in, host_dimg, host_img, host_grads)
    for _ in range(max(1, args.warmup)):
        pipe.submit(host_in, host_dimg, host_img, host_grads)
    pipe.finish()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pipe.submit(host_in, host_dimg, host_img, host_grads)
    pipe.finish()
    t = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
    return {"value": world * px / t / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * t, "api": "render.HostPipeline",
            "serial": {"api": "render.HostStep", "value": world * px / t_serial / 1e6,
                       "ms_per_step": 1e3 * t_serial}}


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
