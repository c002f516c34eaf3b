#!/usr/bin/env python
"""Throughput of the per-frame extraction path (background + detection +
apertures) on the dense 151.2 MP frame (12288 x 12304 uint16, 134,000
sources, mesh 256, 5x5 Gaussian filter, 1.5 sigma, minarea 5, apertures
r = 3, 6, 10).

One step = one gp_extract call on one frame already resident in HBM.  The
frame (302 MB) is larger than L2, so no flush is needed between steps.
Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded crop of the same frame instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpix/s extraction (bkg+detect+aperture) at 151 MP vs roofline; p50/p99 latency"
UNIT = "Mpix/s"
WORKLOAD = "dense_12288x12304_u16"
CAPACITY = 400_000


def env_rank():
    from paper_2609_32375_gb300 import replicas
    return replicas.rank_env()


def workload_config(cfg):
    return {"workload": cfg.name, "width": cfg.width, "height": cfg.height, "dtype_in": cfg.dtype,
            "sources": cfg.nsrc, "mesh": cfg.mesh, "filter": f"{cfg.kernel_size}x{cfg.kernel_size} gaussian "
            f"fwhm {cfg.kernel_fwhm}", "thresh": cfg.thresh, "minarea": cfg.minarea, "radii": list(cfg.radii),
            "l2": "frame (302 MB) larger than the 129 MB L2; no flush between steps"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------ oracle leg ---
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), and its core count."""
    import platform
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    name = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return name or platform.machine(), os.cpu_count() or 1


def oracle_sample(img, cfg, budget_s=12.0, max_crops=6, crop=2048, threads=1, repeats=1):
    """The CPU oracle on crops of the frame until about `budget_s` of CPU
    work, on `threads` host threads (0: every core), best of `repeats` per
    crop; returns (Mpix/s, seconds, description, threads used)."""
    import oracle
    used = oracle.set_threads(threads)
    H, W = img.shape
    offs = [(0, 0), (H // 2, W // 2), (H - crop, W - crop), (0, W - crop), (H - crop, 0), (H // 4, W // 3)]
    tot_px, tot_t, n = 0, 0.0, 0
    try:
        for (y0, x0) in offs[:max_crops]:
            sub = img[y0:y0 + crop, x0:x0 + crop]
            best = None
            for _ in range(repeats):
                t0 = time.perf_counter()
                oracle.extract(sub, cfg.mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain,
                               saturation=cfg.saturation)
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            tot_t += best
            tot_px += sub.size
            n += 1
            if tot_t >= budget_s:
                break
    finally:
        oracle.set_threads(1)
    desc = (f"{n} crop(s) of {crop}x{crop} px ({tot_px / 1e6:.1f} Mpix) of the {cfg.name} frame, full oracle "
            f"path (background, filter, threshold, labelling, moments, apertures), {used} thread(s)"
            + (f", best of {repeats} per crop" if repeats > 1 else ""))
    return tot_px / 1e6 / tot_t, tot_t, desc, used


# ---------------------------------------------------------- clock sampler ---
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "sm_min_mhz": min(sm) if sm else None, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- traffic ---
def kernel_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current sources of that kernel (else None: the kernel changed)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(kernel)
        if not e or e.get("workload") != workload:
            return None
        h = hashlib.sha1()
        for src in e["sources"]:
            h.update(open(os.path.join(ROOT, src), "rb").read())
        return float(e["dram_bytes_per_launch"]) if h.hexdigest() == e.get("sources_sha1") else None
    except Exception:
        return None


STAGE_KERNEL = {"box_stats": "k_boxstats_win", "mesh_spline": "k_mesh_all", "threshold": "k_stream",
                "label_tiles": "k_label_tiles", "tile_merge": "k_merge", "label_rank": "k_rank_scan",
                "measure": "k_measure"}
# stages whose time is one main kernel's launch (the others are several
# launches: labelling runs a common and a crowded-tile form, the merge four
# kernels, the rank four); the roofline is reported for the slowest of these
SINGLE_KERNEL_STAGES = ("threshold", "measure", "box_stats")


def algorithmic_bytes(stage, cfg, cat):
    """Algorithmic DRAM bytes of one launch of a stage's main kernel."""
    import numpy as np
    bpp = 2 if cfg.dtype == "u16" else 4
    npix = cfg.width * cfg.height
    if stage == "box_stats":
        return npix * bpp
    if stage == "threshold":
        # frame read once; uint32 map (zero, or the pixel's m at foreground) and packed mask written
        return npix * (bpp + 4) + npix // 8
    if stage == "label_tiles" and cat is not None:
        # at least: the labels of the kept segments' pixels written, their m read back
        return int(cat["npix"].astype(np.int64).sum()) * 8
    if stage == "measure" and cat is not None:
        bw = (cat["xmax"] - cat["xmin"] + 1).astype(np.int64)
        bh = (cat["ymax"] - cat["ymin"] + 1).astype(np.int64)
        ap = int((2 * max(cfg.radii) + 3) ** 2)
        return int((bw * bh).sum()) * (4 + bpp) + len(bw) * ap * bpp
    return None


# ------------------------------------------------------------- reference ---
def run_reference(args):
    import synth
    rank, world, _ = env_rank()
    if rank != 0:
        return 0                  # the oracle runs on rank 0 alone; the other ranks exit without work
    cfg = synth.CONFIGS[args.workload]
    if args.size:
        w, h = (int(v) for v in args.size.lower().split("x"))
        cfg = synth.scaled_config(cfg, w, h)
    img, _ = synth.make_frame(cfg, 0)
    args.ref_crop = min(args.ref_crop, img.shape[0], img.shape[1])
    times = []
    desc = ""
    mpix = 0.0
    used = 1
    for i in range(args.warmup + args.steps):
        v, t, desc, used = oracle_sample(img, cfg, budget_s=0.0, max_crops=1, crop=args.ref_crop, threads=0)
        if i >= args.warmup:
            times.append(t)
            mpix = args.ref_crop * args.ref_crop / 1e6
    tot = sum(times)
    value = mpix * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot / len(times), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "config": workload_config(cfg),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": used, "kind": "oracle",
                             "cpu": cpu_model()[0], "nproc": cpu_model()[1],
                             "sample": desc + "; each step one crop"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- smaller frames ---
def sizes_section(ctx, t_img, cfg, gp, stream, dev, steps, warmup, peak):
    """The same step, device-resident, on crops of the frame at the paper's
    smaller sizes (2048^2 = 4.2 MP, 4096^2 = 16.8 MP, 8192^2 = 67.1 MP, the
    serving classes): Mpix/s and the path's fraction of the copy bandwidth.
    These frames fit (or nearly fit) in L2, so a 256 MB write flushes it
    between steps, and each step is timed by its own event pair."""
    import torch

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    bpp = t_img.element_size()
    out = {}
    for sz in SERVE_SIZES:
        if sz is None:
            continue
        w, h = sz
        crop = t_img[:h, :w].contiguous()
        ccfg = synth_scaled(cfg, w, h)
        cap = max(8192, (w * h) // 512)
        ex = gp.Extractor(ctx, (h, w), crop.dtype, cfg.mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii,
                          cfg.gain, cap, saturation=cfg.saturation, device=dev)
        for _ in range(max(3, warmup)):
            ex.run(crop)
        ctx.sync()
        n, cat = ex.catalog_host()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 255)
            ev[i][0].record(stream)
            ex.run(crop)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.sync()
        ms = sorted(a.elapsed_time(b) for a, b in ev)
        mean_ms = sum(ms) / len(ms)
        pb = w * h * (2 * bpp + 4) + (algorithmic_bytes("measure", ccfg, cat) or 0)
        out[f"{w * h / 1e6:.1f}MP"] = {
            "width": w, "height": h, "segments": n, "value": round(w * h / 1e6 / (mean_ms / 1e3), 2), "unit": UNIT,
            "ms_per_step": round(mean_ms, 4), "p50_ms": round(ms[len(ms) // 2], 4),
            "path_algorithmic_bytes": pb, "path_frac": round(pb / (mean_ms / 1e3) / 1e9 / peak, 4)}
        del ex
    out["note"] = ("crops of the dense frame, L2 flushed by a 256 MB write before every step, "
                   "per-step CUDA events; path bytes = 2 frame reads + uint32 map + aperture footprints")
    return out


def batching_section(ctx, t_img, cfg, gp, stream, dev, steps, warmup, nb=8, side=2048):
    """nb frames of side^2 px (crops of the frame at distinct offsets) extracted
    one call per frame, and in one gp_extract_batch call (every stage one
    launch over all frames, grid y = frame): the fixed per-frame cost that
    batching removes.  L2 flushed by a 256 MB write before every step."""
    import torch

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    H, W = t_img.shape
    offs = [((i * 3 * side) % (W - side), ((i * 5 * side) // 2) % (H - side)) for i in range(nb)]
    crops = [t_img[y:y + side, x:x + side].contiguous() for x, y in offs]
    cap = max(8192, side * side // 512)
    args = (cfg.mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii, cfg.gain, cap)
    one = gp.Extractor(ctx, (side, side), t_img.dtype, *args, saturation=cfg.saturation, device=dev)
    bat = gp.BatchExtractor(ctx, [(side, side)] * nb, t_img.dtype, *args, saturation=cfg.saturation, device=dev)

    def single(counts=None):
        for c in crops:
            one.run(c)
            if counts is not None:
                counts.append(int(one.out["catalog"]["n"].item()))

    def batched(counts=None):
        outs = bat.run(crops)
        if counts is not None:
            counts.extend(int(o["catalog"]["n"].item()) for o in outs)

    res = {}
    for name, fn in (("single_calls", single), ("one_batched_call", batched)):
        for _ in range(max(3, warmup)):
            fn()
        ctx.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 255)
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.sync()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        counts = []
        fn(counts)
        res[name] = {"ms_per_step": round(ms, 4), "ms_per_frame": round(ms / nb, 4),
                     "value": round(nb * side * side / 1e6 / (ms / 1e3), 2), "unit": UNIT, "segments": counts}
    res["same_segment_counts"] = res["single_calls"]["segments"] == res["one_batched_call"]["segments"]
    res["frames"] = f"{nb} crops of {side}x{side} px at distinct offsets"
    return res


def synth_scaled(cfg, w, h):
    import synth
    return synth.scaled_config(cfg, w, h)


# ---------------------------------------------------------- growth curves ---
def growth_section(ctx, ex, t_img, cfg, nsrc, stream, dev, steps, peak):
    """gp_growth at every catalog centroid with the paper's integer radii,
    ceil(0.75 FWHM) .. ceil(5 FWHM) (Section 3.4), FWHM the frame's PSF
    width.  Kernel time from the context's stage events; bytes are the
    pixels under the largest top-hat, once per source."""
    import numpy as np
    import torch
    fwhm = float(np.mean(cfg.fwhm))
    radii = np.arange(int(np.ceil(0.75 * fwhm)), int(np.ceil(5.0 * fwhm)) + 1, dtype=np.int32)
    n = min(nsrc, CAPACITY)
    xs = ex.out["catalog"]["x"][:n]
    ys = ex.out["catalog"]["y"][:n]
    bkg = {"bkg_mesh": ex.out["bkg_mesh"], "rms_mesh": ex.out["rms_mesh"], "mesh": cfg.mesh}
    for _ in range(3):
        ctx.gp_growth(t_img, bkg, xs, ys, radii, gain=cfg.gain, saturation=cfg.saturation)
    ctx.sync()
    ctx.set_timing(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ctx.gp_growth(t_img, bkg, xs, ys, radii, gain=cfg.gain, saturation=cfg.saturation)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ctx.sync()
    st = ctx.stats()
    ctx.set_timing(False)
    kms = st["ms"]["measure"] / max(st["calls"], 1)
    rmax = int(radii[-1])
    pix = sum(1 for u in range(-rmax, rmax + 1) for v in range(-rmax, rmax + 1) if u * u + v * v <= rmax * rmax)
    nbytes = n * pix * (2 if cfg.dtype == "u16" else 4) + n * len(radii) * 20
    return {"sources": n, "radii": [int(radii[0]), rmax], "nr": int(len(radii)), "fwhm": fwhm,
            "kernel": "k_growth", "kernel_ms": round(kms, 4), "call_ms": round(a.elapsed_time(b) / steps, 4),
            "pixels_per_source": pix, "algorithmic_bytes": nbytes,
            "achieved_GBs": round(nbytes / (kms / 1e3) / 1e9, 1),
            "frac_of_hbm": round(nbytes / (kms / 1e3) / 1e9 / peak, 4),
            "sources_per_s": round(n / (kms / 1e3), 1)}


def timed_calls(ctx, fn, steps, stream, dev):
    """Mean call time (CUDA events) and per-stage device times of `steps` calls."""
    import torch
    for _ in range(3):
        fn()
    ctx.sync()
    ctx.set_timing(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        r = fn()
    b.record(stream)
    torch.cuda.synchronize(dev)
    ctx.sync()
    st = ctx.stats()
    ctx.set_timing(False)
    return a.elapsed_time(b) / steps, {k: v / max(st["calls"], 1) for k, v in st["ms"].items()}, r


def ropt_section(ctx, ex, t_img, cfg, stream, dev, steps):
    """gp_optimal_radius over the catalog: growth curves at the paper's radii,
    nu, calibrators (S/N >= 20, no centroid within 2 r_max), the fit, every
    row's radius (Section 3.4)."""
    import numpy as np
    fwhm = float(np.mean(cfg.fwhm))
    radii = np.arange(int(np.ceil(0.75 * fwhm)), int(np.ceil(5.0 * fwhm)) + 1, dtype=np.int32)
    bkg = {"bkg_mesh": ex.out["bkg_mesh"], "rms_mesh": ex.out["rms_mesh"], "mesh": cfg.mesh}
    cat = ex.out["catalog"]
    ms, stg, out = timed_calls(ctx, lambda: ctx.gp_optimal_radius(t_img, bkg, cfg.kernel, cat, radii, gain=cfg.gain,
                                                                  snr_min=20.0, d_iso=2.0 * float(radii[-1]),
                                                                  saturation=cfg.saturation), steps, stream, dev)
    fit = out["fit"].cpu().numpy()
    return {"rows": int(cat["n"].item()), "radii": [int(radii[0]), int(radii[-1])], "call_ms": round(ms, 4),
            "kernels_ms": round(stg["measure"], 4), "calibrators": int(fit[2]), "a": float(fit[0]),
            "b": float(fit[1]), "snr_min": 20.0, "d_iso": 2.0 * float(radii[-1])}


def psf_section(ctx, ex, t_img, cfg, stream, dev, steps, peak):
    """gp_detect_psf, the second detection pass with a spatially varying PSF
    (Section 3.2), on the same frame: a 13 x 13 Gaussian reference (the
    paper's smallest stamp, half-side 6) and 5 modes, coefficients on
    2048-pixel tiles.  The model is synthetic (the Eigen-PSF stage is out of
    scope), seeded."""
    import numpy as np
    import torch
    H, W = t_img.shape
    size, K, tile = 13, 5, 2048
    h = size // 2
    yy, xx = np.mgrid[-h:h + 1, -h:h + 1].astype(np.float64)
    s = float(np.mean(cfg.fwhm)) / 2.3548
    g = np.exp(-(xx * xx + yy * yy) / (2 * s * s))
    p0 = (g / g.sum()).astype(np.float32)
    r2 = xx * xx + yy * yy
    modes = np.array([xx * p0, yy * p0, (r2 - 2 * s * s) * p0, (xx * xx - yy * yy) * p0, xx * yy * p0], np.float32)
    rng = np.random.default_rng(7)
    coef = torch.from_numpy(rng.uniform(-0.3, 0.3, (K, -(-H // tile), -(-W // tile))).astype(np.float32)).to(dev)
    bkg = {"bkg_mesh": ex.out["bkg_mesh"], "rms_mesh": ex.out["rms_mesh"], "mesh": cfg.mesh}
    ms, stg, out = timed_calls(ctx, lambda: ctx.gp_detect_psf(t_img, bkg, p0, modes, coef, tile, cfg.thresh,
                                                              cfg.minarea, CAPACITY, saturation=cfg.saturation),
                               steps, stream, dev)
    kms = stg["threshold"]
    bpp = 2 if cfg.dtype == "u16" else 4
    nbytes = W * H * (bpp + 4) + W * H // 8
    flops = 2.0 * W * H * (K + 1) * size * size
    return {"model": f"P0 {size}x{size} + {K} modes, tile {tile}", "segments": int(out["catalog"]["n"].item()),
            "call_ms": round(ms, 4), "stages_ms": {k: round(v, 4) for k, v in stg.items()},
            "kernel": "k_psf", "kernel_ms": round(kms, 4), "algorithmic_bytes": nbytes,
            "achieved_GBs": round(nbytes / (kms / 1e3) / 1e9, 1), "frac_of_hbm": round(nbytes / (kms / 1e3) / 1e9 / peak, 4),
            "fp32_tflops": round(flops / (kms / 1e3) / 1e12, 2)}


def deblend_section(ctx, ex, t_img, cfg, stream, dev, steps):
    """gp_deblend on the extraction's segmentation (32 levels, contrast
    0.005), each call on a fresh copy of the map."""
    bkg = {"bkg_mesh": ex.out["bkg_mesh"], "rms_mesh": ex.out["rms_mesh"], "mesh": cfg.mesh}
    seg = ex.out["segmap"].clone()

    def call():
        seg.copy_(ex.out["segmap"])
        return ctx.gp_deblend(t_img, bkg, cfg.kernel, cfg.thresh, cfg.minarea, seg, ex.out["catalog"],
                              saturation=cfg.saturation)
    ms, stg, out = timed_calls(ctx, call, steps, stream, dev)
    c = out["counts"].cpu().numpy()
    return {"segments": int(ex.out["catalog"]["n"].item()), "segments_split": int(c[0]), "objects": int(c[1]),
            "call_ms": round(ms, 4), "kernels_ms": round(stg["measure"], 4), "nthresh": 32, "mincont": 0.005,
            "note": "call_ms includes the copy of the map (604 MB) that gives each call a fresh input"}


def cosmetic_section(ctx, t_img, cfg, stream, dev, steps, peak):
    """gp_cosmetic on the same frame, each filter alone (Section 3.1): the
    cosmic-ray filter (gain and read noise of the frame's recipe) and the
    salt-and-pepper filter (threshold 150.5 ADU)."""
    H, W = t_img.shape
    bpp = 2 if cfg.dtype == "u16" else 4
    nbytes = W * H * (bpp + 4 + 1)          # frame read; float32 frame and flags written
    res = {}
    for name, kw in (("cosmic_ray", dict(cr_gain=cfg.gain, cr_read_noise=3.0)), ("salt_pepper", dict(rtn_t=150.5))):
        ms, _, out = timed_calls(ctx, lambda: ctx.gp_cosmetic(t_img, **kw), steps, stream, dev)
        c = out["counts"].cpu().numpy()
        res[name] = {"call_ms": round(ms, 4), "pixels_changed": int(c[1] if name == "cosmic_ray" else c[0]),
                     "achieved_GBs": round(nbytes / (ms / 1e3) / 1e9, 1),
                     "frac_of_hbm": round(nbytes / (ms / 1e3) / 1e9 / peak, 4)}
    return res


# --------------------------------------------------------------- serving ---
# Frame classes of the request stream: the paper's 4.2 to 151.2 MP range as
# crops of the dense frame (its source density, so 3,700 to 134,000 sources).
SERVE_SIZES = ((2048, 2048), (4096, 4096), (8192, 8192), None)      # None: the whole frame


def serve_stream(srv, frames, caps, arrivals):
    """Submit frames[i] at arrivals[i] seconds (host clock) while a collector
    thread waits for each result and releases it; returns per-request records
    and the server's report for the run."""
    import threading

    n = len(frames)
    tickets = [None] * n
    ready = [threading.Event() for _ in range(n)]
    recs = [None] * n

    def collect():
        for i in range(n):
            ready[i].wait()
            r = srv.wait(tickets[i])
            recs[i] = {"status": r.status, "n": r.n, "latency_ms": r.latency_ms, "queue_ms": r.queue_ms,
                       "batch": r.batch, "mpix": frames[i].shape[0] * frames[i].shape[1] / 1e6,
                       "h2d_ms": r.h2d_ms, "run_ms": r.run_ms, "d2h_ms": r.d2h_ms}
            srv.release(tickets[i])

    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    for i in range(n):
        dt = t0 + arrivals[i] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets[i] = srv.submit(frames[i], caps[i])
        ready[i].set()
    th.join()
    return recs, srv.stats(reset=True)


def _pct(v, q):
    v = sorted(v)
    return v[max(0, min(len(v) - 1, int(-(-q * len(v) // 1)) - 1))]


def summarize(recs, rep, rate):
    lat = [r["latency_ms"] for r in recs if r["status"] == 0]
    by, parts = {}, {}
    for r in recs:
        k = f"{r['mpix']:.1f}MP"
        by.setdefault(k, []).append(r["latency_ms"])
        parts.setdefault(k, []).append((r["queue_ms"], r["h2d_ms"], r["run_ms"], r["d2h_ms"]))
    return {"rate_hz": rate, "requests": len(recs), "ok": len(lat), "p50_ms": round(_pct(lat, 0.5), 3),
            "p99_ms": round(_pct(lat, 0.99), 3), "mean_ms": round(sum(lat) / len(lat), 3),
            "mpix_s": round(rep["mpix"] / rep["wall_s"], 1) if rep["wall_s"] > 0 else None,
            "units": rep["units"], "batched_frames": rep["batched_frames"], "peak_inflight": rep["peak_inflight"],
            "peak_gb": round(rep["peak_bytes"] / 1e9, 2),
            "p50_ms_by_size": {k: round(_pct(v, 0.5), 3) for k, v in sorted(by.items())},
            # median queue wait, input copy, pipeline and result copy by size (device clock for the last three)
            "parts_ms_by_size": {k: [round(_pct([x[i] for x in v], 0.5), 3) for i in range(4)]
                                 for k, v in sorted(parts.items())}}


def serving_section(h_img, cfg, net, gp, seed=0, n_base=24):
    """The request stream at 4 frames/s, a sweep of doubling arrival rates
    until p99 latency diverges, and a closed loop (all requests at once)."""
    import numpy as np
    import synth

    H, W = h_img.shape
    classes = []
    for sz in SERVE_SIZES:
        w, h = (W, H) if sz is None else sz
        classes.append(h_img[:h, :w])
    caps = [max(8192, (c.shape[0] * c.shape[1]) // 512) for c in classes]
    rng = np.random.default_rng(seed)

    def stream(n):
        idx = np.array([i % len(classes) for i in range(n)])
        rng.shuffle(idx)
        return [classes[i] for i in idx], [caps[i] for i in idx]

    srv = gp.Server(device=torch_device_index(), hbm_budget=48 << 30, host_budget=4 << 30, slots=4,
                    batch_pixels=8 << 20, max_batch=8, mesh=cfg.mesh, filter_size=cfg.filter_size,
                    clip_k=cfg.clip_k, clip_maxiter=cfg.clip_maxiter, kernel=cfg.kernel, thresh=cfg.thresh,
                    minarea=cfg.minarea, radii=cfg.radii, gain=cfg.gain, net=net)
    try:
        # cold: the first request of each class on a fresh server, one at a time
        cold = {}
        for c, cap in zip(classes, caps):
            recs, _ = serve_stream(srv, [c], [cap], [0.0])
            cold[f"{c.shape[0] * c.shape[1] / 1e6:.1f}MP"] = round(recs[0]["latency_ms"], 3)
        fr, cp = stream(n_base)
        clk = ClockSampler(torch_device_index())
        clk.start()
        recs, rep = serve_stream(srv, fr, cp, synth.poisson_arrivals(rng, 4.0, n_base))
        base = summarize(recs, rep, 4.0)
        base["clocks"] = clk.stop()          # the GPU idles between requests at this rate
        sweep = [base]
        rate = 8.0
        while rate <= 2048:
            n = int(min(96, max(n_base, rate)))
            fr, cp = stream(n)
            recs, rep = serve_stream(srv, fr, cp, synth.poisson_arrivals(rng, rate, n))
            sweep.append(summarize(recs, rep, rate))
            if sweep[-1]["p99_ms"] > 5 * base["p99_ms"]:
                break                                 # diverged
            rate *= 2
        fr, cp = stream(64)
        recs, rep = serve_stream(srv, fr, cp, [0.0] * 64)
        closed = summarize(recs, rep, None)
    finally:
        srv.close()
    sustained = [s for s in sweep if s["p99_ms"] <= 5 * base["p99_ms"]]
    return {"stream": "Poisson 4 frames/s, equal mix of 4.2/16.8/67.1/151.2 MP crops of the dense frame, uint16, "
                      "in pinned host memory",
            "slots": 4, "hbm_budget_gb": 48, "batch_pixels": 8 << 20, "max_batch": 8,
            "p50_ms": base["p50_ms"], "p99_ms": base["p99_ms"], "mpix_s_at_4hz": base["mpix_s"],
            "cold_ms": cold, "sweep": sweep, "closed_loop": closed,
            "max_sustained": max(sustained, key=lambda s: s["rate_hz"]) if sustained else None}


def torch_device_index():
    import torch
    return torch.cuda.current_device()


# ------------------------------------------------------------------- GPU ---
def run_gpu(args):
    import numpy as np
    import torch

    import paper_2609_32375_gb300 as gp
    import synth

    from paper_2609_32375_gb300 import replicas

    rank, world, local = replicas.rank_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = replicas.init(world, "nccl", dev)
    cfg = synth.CONFIGS[args.workload]
    if args.size:
        w, h = (int(v) for v in args.size.lower().split("x"))
        cfg = synth.scaled_config(cfg, w, h)
    img, _ = synth.make_frame(cfg, replicas.frame_seed(rank))     # one independent frame per rank
    H, W = img.shape
    t_img = torch.from_numpy(img).to(dev)
    L = gp.load_library()
    # the extraction's workspace, and room for the optional steps measured after it (deblending scratch)
    ws = L.gp_workspace_bytes(W, H, cfg.mesh, CAPACITY) + (1 << 30)
    ctx = gp.Context(local, workspace_bytes=ws)
    ex = gp.Extractor(ctx, (H, W), t_img.dtype, cfg.mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii,
                      cfg.gain, CAPACITY, saturation=cfg.saturation, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        ex.run(t_img)
    ctx.sync()
    nsrc, cat = ex.catalog_host()

    # ---- device-resident timed region (no per-stage events inside it: they
    # would sit between the stages' kernels and stall the programmatic
    # launches there; the stage times are taken in a second pass below)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    replicas.barrier(dist)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        ex.run(t_img)
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    replicas.barrier(dist)
    clk = clocks.stop()
    ctx.sync()
    total_ms = t0.elapsed_time(t1)
    # ---- per-stage device times: the same steps again, with an event pair
    # around every stage
    ctx.set_timing(True)
    for i in range(args.steps):
        ex.run(t_img)
    ctx.sync()
    stats = ctx.stats()
    ctx.set_timing(False)
    step_ms = sorted(a.elapsed_time(b) for a, b in ev)
    total_ms = replicas.max_over_ranks(total_ms, dist, dev)
    ms_per_step = total_ms / args.steps
    mpix_all = W * H * world / 1e6
    value = replicas.job_rate(W * H / 1e6, world, ms_per_step / 1e3)

    # ---- end to end from pinned host memory: (a) through the request server,
    # whose slots overlap one frame's copies with another's kernels (the
    # headline e2e), (b) one stream, copy-in / extract / copy-out in sequence
    h_img = torch.from_numpy(img).pin_memory()
    h_frame = h_img                                   # page-locked (cudaHostAlloc) frame for the server paths
    srv = gp.Server(device=local, hbm_budget=24 << 30, host_budget=2 << 30, slots=4, batch_pixels=0, max_batch=1,
                    mesh=cfg.mesh, filter_size=cfg.filter_size, clip_k=cfg.clip_k, clip_maxiter=cfg.clip_maxiter,
                    kernel=cfg.kernel, thresh=cfg.thresh, minarea=cfg.minarea, radii=cfg.radii, gain=cfg.gain)
    srv_d2h = srv.request_bytes(h_frame, CAPACITY)[1]
    for _ in range(max(1, args.warmup // 2)):
        r = srv.result(srv.submit(h_frame, CAPACITY))
        assert r["status"] == 0 and r["n"] == nsrc, "server result differs from the device-resident run"
    srv.stats(reset=True)
    ne2e = args.e2e_steps or args.steps
    replicas.barrier(dist)
    s0 = time.perf_counter()
    tickets = [srv.submit(h_frame, CAPACITY) for _ in range(ne2e)]
    for tk in tickets:
        r = srv.wait(tk)
        assert r.status == 0 and r.n == nsrc, "server result differs from the device-resident run"
        srv.release(tk)
    srv_ms = (time.perf_counter() - s0) * 1e3 / ne2e
    srv_rep = srv.stats()
    srv.close()
    srv_ms = replicas.max_over_ranks(srv_ms, dist, dev)
    ncopy = min(nsrc, CAPACITY)
    nr = len(cfg.radii)
    cat_cols = [v for k, v in ex.out["catalog"].items() if k != "n"]
    h_out = [torch.empty((ncopy,) + tuple(v.shape[1:]), dtype=v.dtype).pin_memory() for v in cat_cols]
    h_ap = [torch.empty((ncopy, ex.out[k].shape[1]), dtype=ex.out[k].dtype).pin_memory()
            for k in ("flux", "fluxerr", "apflags")]
    h_n = torch.empty(1, dtype=torch.int32).pin_memory()
    d2h = h_n.numel() * 4 + sum(t.numel() * t.element_size() for t in h_out + h_ap)
    h2d = h_img.numel() * h_img.element_size()

    def e2e_step():
        t_img.copy_(h_img, non_blocking=True)
        ex.run(t_img)
        h_n.copy_(ex.out["catalog"]["n"], non_blocking=True)
        for src, dst in zip(cat_cols, h_out):
            dst.copy_(src[:ncopy], non_blocking=True)
        for k, dst in zip(("flux", "fluxerr", "apflags"), h_ap):
            dst.copy_(ex.out[k][:ncopy], non_blocking=True)

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    torch.cuda.synchronize(dev)
    replicas.barrier(dist)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(ne2e):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = replicas.max_over_ranks(e0.elapsed_time(e1) / ne2e, dist, dev)
    assert int(h_n.item()) == nsrc, "end-to-end run gave a different segment count"

    # ---- roofline of the dominant kernel (live stage times over the timed region)
    peak, peak_src = measured_peaks()
    stage_ms = {k: v / max(stats["calls"], 1) for k, v in stats["ms"].items()}
    dom = max(SINGLE_KERNEL_STAGES, key=lambda k: stage_ms.get(k, 0.0))
    ab = algorithmic_bytes(dom, cfg, cat)
    achieved = ab / (stage_ms[dom] / 1e3) / 1e9 if ab else None
    roof = {"bound": "hbm", "kernel": STAGE_KERNEL.get(dom, dom), "achieved": round(achieved, 1) if achieved else None,
            "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4) if achieved else None,
            "traffic": kernel_traffic(STAGE_KERNEL.get(dom, dom), cfg.name), "algorithmic_bytes": ab,
            "avg_launch_ms": round(stage_ms[dom], 4), "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}
    path_bytes = W * H * (2 * (2 if cfg.dtype == "u16" else 4) + 4) + (algorithmic_bytes("measure", cfg, cat) or 0)
    whole = {"algorithmic_bytes": path_bytes, "achieved_GBs": round(path_bytes / (ms_per_step / 1e3) / 1e9, 1),
             "frac": round(path_bytes / (ms_per_step / 1e3) / 1e9 / peak, 4)}

    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": dict(workload_config(cfg), parallelism=f"replicas x{world}" if world > 1 else "1 GPU",
                           segments=nsrc, capacity=CAPACITY),
            "p50_ms": round(statistics.median(step_ms), 4),
            "p99_ms": round(step_ms[min(len(step_ms) - 1, int(0.99 * len(step_ms)))], 4),
            "roofline": roof, "path_roofline": whole,
            "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "e2e": {"value": round(mpix_all / (srv_ms / 1e3), 2), "unit": UNIT, "ms_per_step": round(srv_ms, 4),
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": srv_d2h,
                    "path": "gp_server_submit/wait from pinned host memory, 4 slots (copies overlap kernels), "
                            "host clock, whole result block back per frame",
                    "p50_ms": round(srv_rep["p50_ms"], 3), "p99_ms": round(srv_rep["p99_ms"], 3)},
            "e2e_sequential": {"value": round(mpix_all / (e2e_ms / 1e3), 2), "unit": UNIT,
                               "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": h2d,
                               "d2h_bytes_per_step": d2h,
                               "path": "one stream: H2D, gp_extract, D2H of the filled rows, CUDA events"},
            "gpu_launches": stats["launches"] * args.steps,
            "clocks": clk}
    # ---- the same step on the smaller frame sizes of the paper's range
    if not args.no_sizes:
        line["sizes"] = sizes_section(ctx, t_img, cfg, gp, stream, dev, args.steps, args.warmup, peak)
        line["batching"] = batching_section(ctx, t_img, cfg, gp, stream, dev, args.steps, args.warmup)
    # ---- the learned-background form on the same frame (when weights trained
    # at this mesh size are committed)
    from paper_2609_32375_gb300 import learned as L
    wpath = L.weights_for_mesh(cfg.mesh)
    if wpath and not args.no_learned:
        net = L.load(wpath, device=dev)
        exl = gp.Extractor(ctx, (H, W), t_img.dtype, cfg.mesh, cfg.kernel, cfg.thresh, cfg.minarea, cfg.radii,
                           cfg.gain, CAPACITY, saturation=cfg.saturation, device=dev, net=net)
        for _ in range(args.warmup):
            exl.run(t_img)
        ctx.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            exl.run(t_img)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ctx.sync()
        lms = a.elapsed_time(b) / args.steps
        ctx.set_timing(True)                     # stage times in a second pass, as above
        for _ in range(args.steps):
            exl.run(t_img)
        ctx.sync()
        lst = ctx.stats()
        ctx.set_timing(False)
        pb, pr = ex.out["bkg_mesh"], ex.out["rms_mesh"]
        dbk = ((exl.out["bkg_mesh"] - pb) / pr.clamp_min(1e-6)).pow(2).mean().sqrt().item()
        drm = ((exl.out["rms_mesh"] - pr) / pr.clamp_min(1e-6)).pow(2).mean().sqrt().item()
        nl = int(exl.out["catalog"]["n"].item())
        line_learned = {"value": round(mpix_all / (lms / 1e3), 2), "unit": UNIT, "ms_per_step": round(lms, 4),
                        "stages_ms": {k: round(v / max(lst["calls"], 1), 4) for k, v in lst["ms"].items()},
                        "bkg_rmse_vs_plain_sigma": round(dbk, 4), "rms_relerr_vs_plain": round(drm, 4),
                        "segments": nl, "weights": os.path.relpath(wpath, ROOT)}
    else:
        line_learned = None
    if line_learned:
        line["learned"] = line_learned

    # ---- growth curves (top-hat apertures, Section 3.4) at the catalog's centroids
    if not args.no_growth:
        line["growth"] = growth_section(ctx, ex, t_img, cfg, nsrc, stream, dev, args.steps, peak)
        line["optimal_radius"] = ropt_section(ctx, ex, t_img, cfg, stream, dev, args.steps)
        line["psf_detect"] = psf_section(ctx, ex, t_img, cfg, stream, dev, args.steps, peak)
        line["cosmetic"] = cosmetic_section(ctx, t_img, cfg, stream, dev, args.steps, peak)
        line["deblend"] = deblend_section(ctx, ex, t_img, cfg, stream, dev, args.steps)

    # ---- the request server on a mixed stream (plain, and learned when trained weights exist)
    if rank == 0 and world == 1 and not args.no_serving:
        line["serving"] = serving_section(h_frame, cfg, None, gp)
        if line_learned:
            line["serving"]["learned"] = serving_section(h_frame, cfg, net, gp)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on the host's cores: every core (its parallel loops; the
        # labelling stays sequential), and the plain single-threaded definition
        model, nproc = cpu_model()
        va, ta, da, used = oracle_sample(img, cfg, budget_s=6.0, threads=0, repeats=3)
        v1, t1, d1, _ = oracle_sample(img, cfg, budget_s=3.0, max_crops=2, threads=1, repeats=3)
        line["cpu_baseline"] = {"value": round(va, 4), "unit": UNIT, "cores": used, "kind": "oracle",
                                "sample": da, "seconds": round(ta, 2), "cpu": model, "nproc": nproc,
                                "single_thread": {"value": round(v1, 4), "unit": UNIT, "cores": 1, "sample": d1,
                                                  "seconds": round(t1, 2)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    replicas.finish(dist)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--ref-crop", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-background form")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-server stream")
    ap.add_argument("--no-growth", action="store_true", help="skip the growth-curve measurement")
    ap.add_argument("--no-sizes", action="store_true", help="skip the 4.2-67.1 MP frame sizes and the batched small frames")
    ap.add_argument("--size", default=None,
                    help="WxH: run the workload's recipe on a frame of this size (profiling cases)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
