"""Benchmark of the fractal encoder's matching search on one synthetic image
per GPU (512 x 512, 8-bit, seeded; full quadtree 16 -> 8 -> 4 -> 2, domain
step L = 2, RMS split threshold 8, the paper's predefined S per step (Sec.
3.1), entropy threshold at the pool median).

One step = one whole encode (every level: pool, entropy filter, matching,
split) replayed from a captured CUDA graph on an image already resident in
HBM.  The metric is range x domain x isometry matches per second (each match
evaluated over the level's S set), summed over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank encodes its own replica (the workload is
one image; images are independent, nothing is exchanged) and rank 0 prints
the whole-job rate.  `--impl reference` times the CPU oracle instead (rank 0
only), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W_IMG, H_IMG, SEED = 512, 512, 1
METRIC = "range x domain x isometry matches/s (512x512 encode)"
UNIT = "matches/s"
WORKLOAD = ("512x512 8-bit synthetic (seed 1, one textured quadrant), quadtree 16-8-4-2, "
            "L=2, RMS 8, predefined S, median entropy threshold")

# Other workloads (informational runs, --workload): the uneven-size batch and
# the 4096 x 4096 image with the full L = 1 pool.
WORKLOADS = {
    "512": dict(desc=WORKLOAD, metric=METRIC, step=2),
    "batch64": dict(desc=("64 8-bit synthetic images of uneven sizes (seeds 1000-1063, sizes from "
                          "{256x256, 384x512, 512x512, 768x1024, 1024x1024} by a seeded stream, one "
                          "textured tile each), quadtree 16-8-4-2, L=2, RMS 8, predefined S, median "
                          "entropy threshold, one launch per level over all images"),
                    metric="range x domain x isometry matches/s (64-image uneven batch encode)",
                    step=2),
    "4096": dict(desc=("4096x4096 8-bit synthetic (seed 1, 8 textured tiles), quadtree 16-8-4-2, "
                       "L=1 (full pool), RMS 8, predefined S, median entropy threshold"),
                 metric="range x domain x isometry matches/s (4096x4096 L=1 encode)", step=1),
}


def workload_images(name):
    from paper_1501_04140_gb300.synth import batch_specs, synth_image
    if name == "batch64":
        return [synth_image(W, H, sd, n_textured=1) for (W, H, sd) in batch_specs(64, 1000, 42)]
    if name == "4096":
        return [synth_image(4096, 4096, 1, n_textured=8)]
    return [synth_image(W_IMG, H_IMG, SEED, n_textured=1)]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.gpu_id = gpu_identity(index)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "gpu": self.gpu_id}


def gpu_identity(index: int) -> str:
    """nvidia-smi's name for the CUDA device `index`: its UUID (GPU-...), which
    stays right when CUDA_VISIBLE_DEVICES renumbers the devices; the index
    itself when torch cannot tell the UUID."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(index).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    return str(index)


def _sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    except Exception:
        return 2070.0


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_match_tc
# launch per level B on this workload, from one ncu capture of the current
# kernel (cold caches: the operands' first touch); absent (null) when the
# kernel has changed since its last capture.
TRAFFIC = {16: 20139008, 8: 6290688, 4: 3716608, 2: 3509248}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws: int) -> None:
    """All ranks meet here (nothing to do on one rank)."""
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, ws: int, device) -> float:
    """The largest x over the ranks (x itself on one rank): a job is as slow
    as its slowest replica."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(ws: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: the units of every replica over the slowest
    rank's time."""
    return ws * units_per_rank / seconds


# Algorithmic bytes of the HBM-bound steps of one level (summed over the
# images), from the level's counts:
# - pool build (Sec. 3): the images read once; per pool position its entropy
#   key and its two moments written (16 B); per kept domain its index (4 B),
#   its operand row (2 K_p B, f16) and its scoring records (32 B);
# - the rest of the level chain: per active range its pixels (n B) and its
#   domain's (4n B) read, its 8 operand rows written (16 K_p B), and about
#   300 B of moments, candidates, the map and the split's records.
def _kp(B):
    return max(16, B * B)


def pool_bytes(B, s, px_total):
    return float(px_total + 16 * s["pool_size_total"] + s["n_kept"] * (4 + 2 * _kp(B) + 32))


def chain_bytes(B, s):
    return float(s["n_active"] * (5 * B * B + 16 * _kp(B) + 300))


def oracle_extrapolated(img, stats, n_ranges, smode):
    """The oracle on the first n_ranges level-1 ranges of the 4096 x 4096
    workload (the whole level-1 kept pool, a bounded slice of it per call),
    timed and extrapolated linearly to every match of the encode: labelled
    "extrapolated"."""
    import oracle
    cores = os.cpu_count() or 1
    B = stats[0]["size"]
    _, kept, _, _ = oracle.pool_filter(img, B, 1, 0.5)
    sp, q = oracle.s_set(1 if smode else 0, smode.get("grid_samples", 16), B)
    H, W = img.shape
    xy = np.array([(x, y) for y in range(0, H, B) for x in range(0, W, B)][:n_ranges], np.int32)
    t0 = time.perf_counter()
    for c0 in range(0, len(kept), 1 << 19):
        oracle.match(img, B, 1, kept[c0:c0 + (1 << 19)], xy, sp, q, n_threads=cores)
    dt = time.perf_counter() - t0
    rate = len(xy) * len(kept) * 8 / dt
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "extrapolated": True,
            "sample": f"first {len(xy)} level-1 ranges x {len(kept)} kept domains x 8 in "
                      f"{dt:.1f}s, extrapolated to the encode's matches at that rate",
            "encode_s_extrapolated": sum(s["matches"] for s in stats) / rate,
            "cpu_model": _cpu_model()}


def measure_batch64(ctx, stream, l2_flush, steps=3, warmup=3):
    """Encode time of the 64-image uneven batch (graph replay, CUDA events,
    L2 flushed between steps): matches/s and ms per batch and per image."""
    import torch
    from paper_1501_04140_gb300 import fic
    imgs = workload_images("batch64")
    d = [torch.from_numpy(im).cuda() for im in imgs]
    p = fic.default_params()
    code = ctx.encode(d, p, stream=stream)
    torch.cuda.synchronize()
    matches = sum(sum(s["matches"] for s in code.stats(i)) for i in range(len(imgs)))
    for _ in range(warmup):
        ctx.encode_again(code, d, p, stream=stream)
    times = []
    for _ in range(steps):
        l2_flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.encode_again(code, d, p, stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    code.free()
    ms = statistics.mean(times)
    return {"workload": WORKLOADS["batch64"]["desc"], "value": matches / (ms * 1e-3),
            "unit": UNIT, "ms_per_batch": ms, "ms_per_image": ms / len(imgs),
            "n_images": len(imgs), "matches_per_batch": matches, "steps": steps,
            "warmup": warmup}


# ------------------------------------------------------------------ oracle
def oracle_rate(img, level_stats, budget_s: float, n_threads: int):
    """The oracle's matches/s on a bounded sample: per level, the exhaustive
    search for a few ranges against the level's kept pool, timed; the
    level's rate is applied to that level's share of the workload."""
    import oracle
    total_m = 0.0
    total_t = 0.0
    sample = []
    per_level = budget_s / max(1, len(level_stats))
    for lv, st in enumerate(level_stats):
        B = st["size"]
        if st["n_active"] == 0:
            continue
        _, kept, _, _ = oracle.pool_filter(img, B, 2, 0.5)
        sp, q = oracle.s_set(0, 16, B)
        xs = [(x, y) for y in range(0, H_IMG, B) for x in range(0, W_IMG, B)]
        k = max(1, n_threads)
        t_used = 0.0
        done = 0
        rng = np.random.default_rng(lv)
        while t_used < per_level and done < len(xs):
            pick = np.array([xs[i] for i in rng.choice(len(xs), size=k, replace=False)], np.int32)
            t0 = time.perf_counter()
            oracle.match(img, B, 2, kept, pick, sp, q, n_threads=n_threads)
            t_used += time.perf_counter() - t0
            done += k
            k *= 2
        rate = done * len(kept) * 8 / t_used
        total_m += st["matches"]
        total_t += st["matches"] / rate
        sample.append(f"B={B}: {done} ranges x {len(kept)} domains x 8 in {t_used:.1f}s")
    return total_m / total_t, "; ".join(sample)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_1501_04140_gb300.synth import synth_image
    img = synth_image(W_IMG, H_IMG, SEED, n_textured=1)
    cores = os.cpu_count() or 1
    # the workload's per-level match counts, from the oracle's own pools and
    # the level-1 range grid (later levels: the counts the GPU encode reports
    # are not used here; each step samples level 1 of the search)
    _, kept, _, _ = oracle.pool_filter(img, 16, 2, 0.5)
    sp, q = oracle.s_set(0, 16, 16)
    xs = np.array([(x, y) for y in range(0, H_IMG, 16) for x in range(0, W_IMG, 16)], np.int32)
    per_step = max(cores, 16)
    rates = []
    for s in range(args.warmup + args.steps):
        pick = xs[(s * per_step) % len(xs):][:per_step]
        t0 = time.perf_counter()
        oracle.match(img, 16, 2, kept, pick, sp, q, n_threads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            rates.append(len(pick) * len(kept) * 8 / dt)
    v = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64 (exact)",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "level-1 ranges"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} level-1 ranges per step vs {len(kept)} kept "
                                   f"domains x 8 isometries", "cpu_model": _cpu_model()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ tables
def run_tables(args):
    """Tables 1-2's layout on synthetic stand-ins (the paper's Baboon / F16
    are not reproduced): for pool sizes 256, 64 and 32, the proposed method
    (Sec. 3.1's predefined S) against the entropy-only baseline (a 10-sample s
    grid), each with the encode time (GPU, graph replay, median of steps),
    the compression ratio of the stored form (o in 7 bits) and the PSNR of its
    decoded image."""
    import torch
    from paper_1501_04140_gb300 import build, fic
    build.build()
    import oracle
    from paper_1501_04140_gb300.synth import synth_image
    ctx = fic.Context(0)
    stream = torch.cuda.Stream()
    images = {"smooth+edges 512 (seed 3)": synth_image(512, 512, 3, n_textured=0),
              "textured 512 (seed 1)": synth_image(512, 512, 1, n_textured=1)}
    rows = []
    for name, img in images.items():
        d = torch.from_numpy(img).cuda()
        for K in (256, 64, 32):
            for method, kw in (("proposed (predefined S)", dict(s_mode=fic.FIC_S_PREDEFINED)),
                               ("entropy-based (10-sample s grid)",
                                dict(s_mode=fic.FIC_S_GRID, grid_samples=10))):
                p = fic.default_params(pool_size=K, **kw)
                code = ctx.encode(d, p, stream=stream)
                times = []
                for s_ in range(args.warmup + args.steps):
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ctx.encode_again(code, d, p, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                    if s_ >= args.warmup:
                        times.append(e0.elapsed_time(e1))
                bits = code.bits(0, 7)
                code.quantize_o(7)
                psnr = oracle.psnr(img, code.decode(0))
                rows.append({"image": name, "pool_size": K, "method": method,
                             "encode_ms": statistics.median(times),
                             "compression_ratio": 8.0 * img.size / bits, "psnr_db": psnr,
                             "n_maps": code.count(0)})
                code.free()
    print(json.dumps({"workload": "tables", "rows": rows}))
    return 0


def _cpu_model():
    """The host CPU's model name from /proc/cpuinfo (else the machine type)."""
    import platform
    part = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip().lower() in ("model name", "cpu model", "hardware"):
                    return v.strip()
                if k.strip().lower() == "cpu part" and part is None:
                    part = v.strip()
    except OSError:
        pass
    return platform.machine() + (f" (CPU part {part})" if part else "")


# ------------------------------------------------------------------ s histogram
def _kmeans_1d(x, k, iters=50):
    """Lloyd's k-means on the line from the quantile starts (k = 1: the mean)."""
    import numpy as np
    c = np.quantile(x, [(i + 0.5) / k for i in range(k)])
    for _ in range(iters):
        lab = np.argmin(np.abs(x[:, None] - c[None, :]), axis=1)
        c = np.array([x[lab == i].mean() if np.any(lab == i) else c[i] for i in range(k)])
    return np.sort(c)


def run_shist(args):
    """Fig. 3's study on synthetic stand-ins (the paper's test images are not
    reproduced): a batch of 512x512 images encoded with an exhaustive s
    search -- Eq. 2's s of every pair (FIC_S_EXACT) and the 10-sample grid of
    the "existing algorithms" -- and, per quadtree step, the histogram of the
    s of the saved maps (10 bins over [0, 1]).  Sec. 3.1 reads its predefined
    sets off such histograms (one value at step 1, two below); the rule here
    is 1-D k-means of the exact-s values (k = 1 at step 1, 2 below) rounded
    to 0.1.  Also times each encode (GPU, graph replay) and the PSNR."""
    import numpy as np
    import torch
    from paper_1501_04140_gb300 import build, fic
    build.build()
    import oracle
    from paper_1501_04140_gb300.synth import synth_image
    ctx = fic.Context(0)
    stream = torch.cuda.Stream()
    imgs = [synth_image(512, 512, seed, n_textured=seed % 2) for seed in range(1, 9)]
    dev = [torch.from_numpy(i).cuda() for i in imgs]
    out = {"workload": "s histogram (Fig. 3) on 8 synthetic 512x512 images, L = 2, RMS 8",
           "modes": {}}
    for name, kw in (("exact s (Eq. 2, clamped)", dict(s_mode=fic.FIC_S_EXACT)),
                     ("10-sample grid", dict(s_mode=fic.FIC_S_GRID, grid_samples=10)),
                     ("predefined (Sec. 3.1)", dict(s_mode=fic.FIC_S_PREDEFINED))):
        p = fic.default_params(**kw)
        code = ctx.encode(dev, p, stream=stream)
        times = []
        for s_ in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.encode_again(code, dev, p, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if s_ >= args.warmup:
                times.append(e0.elapsed_time(e1))
        per_level = [[] for _ in range(4)]
        psnr = []
        for i, img in enumerate(imgs):
            t = code.transforms(i)
            for lv in range(4):
                per_level[lv].extend(t["s"][t["level"] == lv].tolist())
            psnr.append(oracle.psnr(img, code.decode(i)))
        levels = []
        for lv, vals in enumerate(per_level):
            v = np.asarray(vals)
            h, _ = np.histogram(v, bins=10, range=(0.0, 1.0))
            row = {"step": lv + 1, "B": 16 >> lv, "n_maps": int(v.size), "hist_10_bins": h.tolist(),
                   "median_s": float(np.median(v)) if v.size else None}
            if kw["s_mode"] == fic.FIC_S_EXACT and v.size:
                c = _kmeans_1d(v, 1 if lv == 0 else 2)
                row["derived_set"] = [round(float(min(max(x, 0.1), 0.9)), 1) for x in c]
            levels.append(row)
        out["modes"][name] = {"encode_ms_per_batch": statistics.median(times),
                              "mean_psnr_db": float(np.mean(psnr)), "levels": levels}
        code.free()
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ decode
def run_decode(args):
    """Decoder throughput: the 512x512 headline image's saved maps decoded
    from a flat 128 image to the fixed point (FP64 Jacobi steps until max
    |delta| < 1e-7, then rounding) into device memory, timed with CUDA events
    per decode; reports decoded images/s and pixel-iterations/s."""
    import torch
    from paper_1501_04140_gb300 import build, fic
    build.build()
    import oracle
    from paper_1501_04140_gb300.synth import synth_image
    ctx = fic.Context(0)
    img = synth_image(512, 512, 1, n_textured=1)
    d = torch.from_numpy(img).cuda()
    code = ctx.encode(d, fic.default_params())
    out = torch.zeros((512, 512), dtype=torch.uint8, device="cuda")
    times, iters = [], 0
    for s_ in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        code.decode(0, out=out)
        e1.record()
        e1.synchronize()
        iters = code.iters
        if s_ >= args.warmup:
            times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    psnr = oracle.psnr(img, out.cpu().numpy())
    line = {"metric": "decoded images/s (512x512, to the fixed point)", "value": 1e3 / ms,
            "unit": "images/s", "higher_is_better": True, "ms_per_decode": ms,
            "iterations": iters, "pixel_iterations_per_s": 512 * 512 * iters / (ms * 1e-3),
            "n_maps": code.count(0), "psnr_db": psnr, "steps": args.steps,
            "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": "decode of the 512x512 encode (seed 1, one textured quadrant)"}}
    code.free()
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ ours
def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1501_04140_gb300 import build, fic
    build.build()
    from paper_1501_04140_gb300.synth import synth_image
    import oracle

    wl = WORKLOADS[args.workload]
    imgs = workload_images(args.workload)
    img = imgs[0]
    ctx = fic.Context(local)
    stream = torch.cuda.Stream()
    d_imgs = [torch.from_numpy(im).cuda() for im in imgs]
    d_img = d_imgs if len(d_imgs) > 1 else d_imgs[0]
    l2_flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    smode = dict(s_mode=fic.FIC_S_GRID, grid_samples=int(args.smode[4:])) \
        if args.smode.startswith("grid") else {}

    def time_path(precision, steps, warmup, profile=False, prof_steps=None):
        """Headline steps with no timing events inside the encode (events
        between the level chain's kernels would cut their programmatic
        launch overlap); then, if profile, a second pass with the per-level
        events captured into the graph for the breakdown."""
        p = fic.default_params(precision=precision, domain_step=wl["step"],
                               autotune=1 if args.autotune else 0, **smode)
        with torch.cuda.stream(stream):
            code = ctx.encode(d_img, p, stream=stream)
        torch.cuda.synchronize()
        # per level, summed over the images
        per_img = [code.stats(i) for i in range(len(imgs))]
        stats = []
        for lv in range(len(per_img[0])):
            agg = dict(per_img[0][lv])
            for k in ("n_active", "n_kept", "matches"):
                agg[k] = sum(ps[lv][k] for ps in per_img)
            agg["pool_size_total"] = sum(ps[lv]["pool_size"] for ps in per_img)
            stats.append(agg)
        for _ in range(warmup):
            ctx.encode_again(code, d_img, p, stream=stream)
        torch.cuda.synchronize()
        times = []
        _barrier(ws)
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            for _ in range(steps):
                l2_flush.zero_()  # inputs are smaller than L2: flush between steps
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.encode_again(code, d_img, p, stream=stream)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        _barrier(ws)
        prof = None
        if profile:
            n_prof = prof_steps if prof_steps is not None else max(3, steps // 2)
            code.set_profiling(True)
            ctx.encode_again(code, d_img, p, stream=stream)  # captures the profiled graph
            torch.cuda.synchronize()
            prof = []
            for _ in range(n_prof):
                l2_flush.zero_()
                torch.cuda.synchronize()
                ctx.encode_again(code, d_img, p, stream=stream)
                try:
                    prof.append([lv + (pm,) for lv, pm in zip(code.profile(),
                                                              code.pool_profile())])
                except fic.FicError as e:  # events inside the graph unusable
                    print(f"in-graph profile failed ({e}); timing kernels outside it",
                          file=sys.stderr)
                    prof = None
                    break
            if prof is None:
                prof = []
                for _ in range(n_prof):
                    l2_flush.zero_()
                    torch.cuda.synchronize()
                    ctx.encode_again(code, d_img, p, stream=None)
                    prof.append([lv + (pm,) for lv, pm in zip(code.profile(),
                                                              code.pool_profile())])
            torch.cuda.synchronize()
        return code, stats, times, prof, clk.summary()

    # exact tensor path: the headline steps, then the per-level breakdown
    code, stats, times, prof, clocks = time_path(fic.FIC_PREC_TENSOR, args.steps, args.warmup,
                                                 profile=True)
    matches = sum(s["matches"] for s in stats)
    ms = statistics.mean(times)
    n_kernels = code.graph_kernels()
    sched = code.schedule()
    dec = code.decode(0)
    psnr = oracle.psnr(img, dec)  # the first image

    # max over ranks
    t_max = _max_over_ranks(ms, ws, "cuda")
    value = _job_rate(ws, matches, t_max * 1e-3)

    # roofline of the dominant kernel: the tensor matcher at its costliest
    # level.  Per match (range x isometry x kept domain) it does 2n MMA flops
    # (tensor pipe).  Its epilogue works per (range, domain) pair of 8
    # matches: 7 two-input maxima over the isometries, then y, one score per
    # s, |S| - 1 minima and one compare, i.e. (8 + 2|S|) / 8 FP32 lane-ops
    # per match.  Whichever needs longer at its peak bounds the level.
    hbm, bf16, peak_kind = _peaks()
    props = torch.cuda.get_device_properties(local)
    sm_mhz = _sm_max_mhz()
    alu_peak = props.multi_processor_count * 128 * sm_mhz * 1e6 / 1e12  # Top/s
    lv_ms = [statistics.mean(p[l][0] for p in prof) for l in range(len(stats))]
    lv_all = [statistics.mean(p[l][1] for p in prof) for l in range(len(stats))]
    lv_pool = [statistics.mean(p[l][2] for p in prof) for l in range(len(stats))]
    px_total = sum(im.size for im in imgs)
    levels = []
    for l, s in enumerate(stats):
        B = s["size"]
        # |S|: the predefined sets of Sec. 3.1, or the grid (whose epilogue
        # scores the 3 grid points around the real minimiser)
        n_s = (1 if B == 16 else 2) if not smode else 3
        flop = 2.0 * B * B * s["matches"]
        ops = (8 + 2 * n_s) / 8.0 * s["matches"]
        sec = lv_ms[l] * 1e-3
        tensor_bound = flop / (bf16 * 1e12) >= ops / (alu_peak * 1e12)
        ach = (flop if tensor_bound else ops) / sec / 1e12 if sec > 0 else 0.0
        pk = bf16 if tensor_bound else alu_peak
        pool_b, other_b = pool_bytes(B, s, px_total), chain_bytes(B, s)
        other_ms = lv_all[l] - lv_ms[l]
        levels.append({"B": B, "n_active": s["n_active"], "n_kept": s["n_kept"],
                       "matches": s["matches"], "matcher_ms": lv_ms[l], "level_ms": lv_all[l],
                       "schedule": {"items_per_cta": sched[l][0],
                                    "groups_per_tile": sched[l][1]},
                       # the level's pool build (side stream) and the rest of its
                       # chain (range operand, plan, reduction, split): HBM-bound
                       # in design; algorithmic bytes over the measured time
                       "pool_ms": lv_pool[l], "pool_bytes": pool_b,
                       "pool_hbm_frac": pool_b / (lv_pool[l] * 1e-3) / (hbm * 1e9)
                       if lv_pool[l] > 0 else 0.0,
                       "chain_ms": other_ms, "chain_bytes": other_b,
                       "chain_hbm_frac": other_b / (other_ms * 1e-3) / (hbm * 1e9)
                       if other_ms > 0 else 0.0,
                       "bound": "tensor" if tensor_bound else "alu",
                       "achieved": ach, "unit": "TFLOP/s" if tensor_bound else "Top/s",
                       "frac": ach / pk if pk else 0.0,
                       "matches_per_s": s["matches"] / sec if sec > 0 else 0.0,
                       # every (range, domain, isometry, s) of the level's set
                       "s_evaluations_per_s": (smode.get("grid_samples", n_s)) * s["matches"] / sec
                       if sec > 0 else 0.0})
    dom = max(range(len(levels)), key=lambda l: levels[l]["matcher_ms"])
    d = levels[dom]
    roofline = {"bound": d["bound"], "achieved": d["achieved"],
                "peak": bf16 if d["bound"] == "tensor" else alu_peak, "unit": d["unit"],
                "frac": d["frac"], "traffic": TRAFFIC.get(d["B"]), "kernel": "k_match_tc",
                "level_B": d["B"],
                "peak_source": (f"{peak_kind} dense bf16 (f16 has the same dense rate)"
                                if d["bound"] == "tensor" else
                                f"FP32 lanes: {props.multi_processor_count} SMs x 128 x "
                                f"{sm_mhz:.0f} MHz (derived)")}

    # plain FP32 CUDA-core path, same workload (not on the 4096 x 4096 run,
    # where one FP32 encode takes minutes)
    fp32 = None
    if args.workload != "4096" or args.fp32_4096:
        # (4096 x 4096: one FP32 encode takes tens of seconds, so one warm-up
        # and one timed encode, stated in the line)
        big = args.workload == "4096"
        fp_steps, fp_warm = (1, 1) if big else (max(3, args.steps // 4), 3)
        code32, stats32, times32, prof32, _ = time_path(fic.FIC_PREC_FP32, fp_steps, fp_warm,
                                                        profile=True,
                                                        prof_steps=1 if big else None)
        ms32 = statistics.mean(times32)
        psnr32 = oracle.psnr(img, code32.decode(0))
        matches32 = sum(s["matches"] for s in stats32)
        code32.free()
        # the FP32 matcher per level: 2n FMA flops per match (its SGEMM of the
        # isometry rows against the domains) against the FP32 FMA roof
        fma_peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
        lv32 = []
        for l, s32 in enumerate(stats32):
            B = s32["size"]
            m_ms = statistics.mean(p[l][0] for p in prof32)
            tf = 2.0 * B * B * s32["matches"] / (m_ms * 1e-3) / 1e12 if m_ms > 0 else 0.0
            lv32.append({"B": B, "matches": s32["matches"], "matcher_ms": m_ms,
                         "level_ms": statistics.mean(p[l][1] for p in prof32),
                         "achieved": tf, "unit": "TFLOP/s", "peak": fma_peak, "frac": tf / fma_peak,
                         "peak_source": f"FP32 FMA: {props.multi_processor_count} SMs x 128 x 2 x "
                                        f"{sm_mhz:.0f} MHz (derived)"})
        fp32 = {"value": matches32 / (ms32 * 1e-3), "unit": UNIT, "encode_ms": ms32,
                "psnr_db": psnr32, "levels": lv32, "steps": fp_steps, "warmup": fp_warm,
                "speedup_tensor_vs_fp32": (matches / (t_max * 1e-3)) / (matches32 / (ms32 * 1e-3))}

    # end to end through the C ABI with host buffers: pinned host images in,
    # every saved map out, both copies inside the timed region
    pinned = [torch.from_numpy(im).pin_memory() for im in imgs]
    ph = pinned if len(pinned) > 1 else pinned[0]
    # the same parameters as the device-timed path (its schedule included:
    # the handle's first encode runs the autotuner when it is on)
    p = fic.default_params(domain_step=wl["step"], autotune=1 if args.autotune else 0, **smode)
    code_h = ctx.encode(ph, p, stream=stream)
    torch.cuda.synchronize()
    n_codes = sum(code_h.count(i) for i in range(len(imgs)))
    # page-locked output buffers, allocated once (room for every 2 x 2 range)
    outs_buf = [torch.empty((im.size // 4) * fic.TRANSFORM_DTYPE.itemsize, dtype=torch.uint8,
                            pin_memory=True).numpy().view(fic.TRANSFORM_DTYPE) for im in imgs]
    e2e = []
    e2e_steps = args.steps if args.workload == "512" else 1
    e2e_warm = args.warmup if args.workload == "512" else 1
    for s in range(e2e_warm + e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.encode_again(code_h, ph, p, stream=stream)
        outs = [code_h.transforms(i, out=outs_buf[i]) for i in range(len(imgs))]
        t1 = time.perf_counter()
        if s >= e2e_warm:
            e2e.append(t1 - t0)
    e2e_v = _job_rate(ws, matches, _max_over_ranks(statistics.mean(e2e), ws, "cuda"))
    # the maps, plus the one read-back of every level's code offsets and the
    # status word
    d2h = (sum(len(o) * o.dtype.itemsize for o in outs)
           + 8 * 4 * (len(imgs) + 1) + 16)
    code_h.free()

    # the 64-image uneven batch, a few graph replays (the same encoder, one
    # launch per step and level over all images)
    batch = None
    if args.workload == "512" and not args.no_batch:
        batch = measure_batch64(ctx, stream, l2_flush, steps=3, warmup=3)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload == "512":
        cores = os.cpu_count() or 1
        v, sample = oracle_rate(img, stats, args.cpu_budget, cores)
        # and single-threaded, the way the paper ran its encoder (Sec. 4)
        v1, sample1 = oracle_rate(img, stats, args.cpu_budget / 2, 1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "cpu_model": _cpu_model(),
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1}}

    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload == "4096":
        cpu = oracle_extrapolated(img, stats, args.oracle_ranges, smode)

    if rank == 0:
        line = {
            "metric": wl["metric"], "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16 MMA on exact integers, int64 scoring",
            "data": "synthetic",
            "config": {"workload": wl["desc"] if not smode else
                       wl["desc"].replace("predefined S", f"{smode['grid_samples']}-sample s grid"),
                       "parallelism": f"replicas x{ws}",
                       "l2": "flushed between steps (256 MB write)",
                       "encode_ms": t_max, "psnr_db": psnr, "n_codes": n_codes,
                       "n_images": len(imgs), "matches_per_step": matches},
            "fp32_path": fp32,
            "batch64": batch,
            "levels": levels,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_v, "unit": UNIT,
                    "h2d_bytes_per_step": sum(im.size for im in imgs),
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": n_kernels * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line))
    code.free()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=16.0,
                    help="seconds of oracle work for the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--smode", default="predefined",
                    help="predefined (Sec. 3.1's sets, the default) or gridM (an M-sample grid)")
    ap.add_argument("--fp32-4096", action="store_true",
                    help="also time the FP32 path on the 4096 x 4096 workload (minutes)")
    ap.add_argument("--oracle-ranges", type=int, default=16,
                    help="4096 workload: level-1 ranges the oracle is timed on (extrapolated)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the short 64-image batch measurement of the default run")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the library's default schedule (by default the library times "
                         "its schedules on the first encode and keeps the fastest)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["tables", "decode", "shist"],
                    default="512",
                    help="512 (the headline), batch64, 4096, tables, decode or shist "
                         "(informational runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "tables":
        return run_tables(args)
    if args.workload == "decode":
        return run_decode(args)
    if args.workload == "shist":
        return run_shist(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
