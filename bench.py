#!/usr/bin/env python
"""Benchmark of the GPSS renderer on GB300: million path vertices per second.

A *path vertex* is one real scattering event of a path (free flight into it,
next-event estimation and phase sampling at it).  One benchmark step is one full
forward render of the workload; the default workload is the surface-to-volume
scene, the largest configuration (torus, box and sphere on their own 256^3 grids,
variances 1e-6 / 2.24e-4 / 0.05, RGB albedo; 1024x1024, 256 spp, 64 bounces, sky
light; about 1 GB of grids, more than L2).  The tiny slab and the heterogeneous
128^3 workload are timed too, as extra keys.

Output: one JSON line (rank 0).  ``value`` is the whole-job throughput with the
scene resident in HBM; ``e2e`` is the same metric through the C-ABI with host
buffers (grids uploaded and the image read back every step); ``roofline`` is
the FP32-issue bound of the render kernel (algorithmic ops from the committed
tally of the formulas, paper_2603_00280_gb300/opcounts.json); ``roofline_hbm``
sets the algorithmic gather bytes against HBM; ``cpu_baseline`` is the FP64
oracle on a bounded sample of the same workload on this machine's cores (and on
one core).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M path-vertices/s at 1 GB300 (fwd; fwd+adjoint) and fraction of FP32-issue roofline"
UNIT = "M path-vertices/s"


def opcounts():
    """Algorithmic FP32 work per unit, tallied from the formulas (not the code): one
    extinction evaluation (field fetch + sigma_t + the tracking step) per tentative
    collision, plus the shading of each real vertex (phase sampling + NEE phase
    evaluation + MIS); and the field bytes one extinction evaluation gathers."""
    from paper_2603_00280_gb300 import opcounts as oc
    t = oc.load()
    return t["ops_per_extinction_evaluation"], t["ops_per_vertex_shading"], t["bytes_per_extinction_evaluation"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["surface_to_volume", "heterogeneous", "tiny_slab"],
                    default="surface_to_volume")
    ap.add_argument("--no-configs", action="store_true", help="skip the extra configurations (tiny slab, 128^3)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--image", type=int, default=0, help="override the image side (profiling of small cases)")
    ap.add_argument("--spp", type=int, default=0, help="override samples per pixel (profiling of small cases)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-vndf", action="store_true", help="skip the exact visible-normal sampler comparison")
    ap.add_argument("--batch-count", type=int, default=64, help="scenes of the batched comparison")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="image/grid size scale of the batched scenes")
    return ap.parse_args()


def workload(name, seed_offset=0, image=0, spp=0):
    from paper_2603_00280_gb300 import workloads as W
    if name == "tiny_slab":
        wl = W.tiny_slab()
    elif name == "surface_to_volume":
        wl = W.surface_to_volume()
    else:
        wl = W.heterogeneous()
    wl["opts"] = dict(wl["opts"], seed=wl["opts"]["seed"] + seed_offset)
    if image:
        wl["camera"] = dict(wl["camera"], width=image, height=image)
        wl["name"] += "_img%d" % image
    if spp:
        wl["opts"]["spp"] = spp
        wl["name"] += "_spp%d" % spp
    return wl


def config_of(wl, l2):
    cam, opts = wl["camera"], wl["opts"]
    objs = wl["scene"]["objects"]
    grids = [list(o["mean"].shape[::-1]) for o in objs]
    nbytes = sum(o["mean"].size * 4 * (2 + (o["albedo"].shape[0] if o["albedo"].ndim == 4 else 1)) for o in objs)
    return {"workload": wl["name"], "objects": len(objs), "grid": grids[0] if len(grids) == 1 else grids,
            "grid_bytes": nbytes, "image": [cam["width"], cam["height"]],
            "spp": opts["spp"], "max_bounces": opts["max_bounces"], "light": wl["scene"]["light"]["type"],
            "l2": l2}


# ----------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ----------------------------------------------------------------- roofline
def peak_fp32_tops(torch):
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    mhz = None
    try:
        mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]
        src = "MEASURED_PEAKS.json sm_max_mhz"
    except Exception:
        src = "nominal 2070 MHz"
        mhz = 2070.0
    return sms * 128 * mhz * 1e6 / 1e12, sms, mhz, src


# The files the measured render kernel (k_path<0, 0, 0>) is built from: its translation
# unit render.cu with every header it includes, and the build script's flags.
KERNEL_SOURCES = ("paper_2603_00280_gb300/csrc/render.cu", "paper_2603_00280_gb300/csrc/path_kernel.cuh",
                  "paper_2603_00280_gb300/csrc/adjoint_math.cuh", "paper_2603_00280_gb300/csrc/gpss_internal.h",
                  "paper_2603_00280_gb300/csrc/gpss_device.cuh", "paper_2603_00280_gb300/csrc/moment_fit.inc",
                  "include/gpss.h", "paper_2603_00280_gb300/build.py")


def strip_comments(src: str) -> str:
    """C/C++ source without its comments and blank lines (string literals in these
    files hold no comment markers): comment edits leave the compiled kernel unchanged."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_source_hash():
    h = hashlib.sha1()
    for rel in KERNEL_SOURCES:
        text = open(os.path.join(ROOT, rel), encoding="utf-8").read()
        h.update((text if rel.endswith(".py") else strip_comments(text)).encode())
    return h.hexdigest()[:12]


def measured_traffic(workload_name):
    """DRAM bytes per launch of the render kernel from a committed ncu summary,
    valid only while the kernel sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))
        e = t[workload_name]
        if e.get("source_hash") == kernel_source_hash():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def evaluations(st):
    """Extinction evaluations of a render: one per tentative collision (real, null, shadow)."""
    return st["vertices"] + st["null_collisions"] + st["shadow_steps"]


def algorithmic_ops(st):
    per_eval, per_vertex, _ = opcounts()
    return per_eval * evaluations(st) + per_vertex * st["vertices"]


# ----------------------------------------------------------------- CPU oracle sample
def oracle_sample(wl, target_seconds, threads=0):
    """Renders a bounded block of pixels of the workload with the FP64 oracle (its
    bounce limit, at most 16 samples per pixel, 4 pixels per row with one row per
    worker thread at a time); returns (vertices/s, description, cores, seconds)."""
    import oracle
    O = oracle.Scene(wl["scene"])
    cam, opts = wl["camera"], wl["opts"]
    H, W = cam["height"], cam["width"]
    cy, cx = H // 2, W // 2
    cores = threads if threads > 0 else (os.cpu_count() or 1)
    spp = min(opts["spp"], 16)
    sopts = dict(opts, spp=spp)
    t0 = time.perf_counter()
    oracle.render(O, cam, sopts, rows=(cy, cy + 1, 1), cols=(cx, cx + 1), threads=1)
    per_px = max(time.perf_counter() - t0, 1e-4)  # one pixel's paths on one thread
    cols = 4
    per_row = per_px * cols
    n_rows = max(1, min(H // 2, int(target_seconds / per_row) * cores))
    step = max(1, (H // 2) // n_rows)
    rows = (H // 4, H // 4 + n_rows * step, step)
    c0, c1 = cx - cols // 2, cx + cols // 2
    t0 = time.perf_counter()
    _, _, st = oracle.render(O, cam, sopts, rows=rows, cols=(c0, c1), threads=threads)
    dt = time.perf_counter() - t0
    desc = "%d pixels (rows %d:%d:%d, cols %d:%d) x %d spp, %d paths, %d vertices, %.1f s on %d thread(s)" % (
        n_rows * cols, rows[0], rows[1], rows[2], c0, c1, spp, st["paths"], st["vertices"], dt, cores)
    return st["vertices"] / dt / 1e6, desc, cores, dt


# ----------------------------------------------------------------- ranks
def job_totals(total_ms, units, dist=None, device="cpu"):
    """Whole-job totals over ranks: the slowest rank's time (max) and the units
    all ranks processed (sum).  Weak scaling: every rank renders the full
    workload with its own random numbers, so the ranks exchange nothing but these two
    numbers (each rank keys its paths with seed + 1000 * rank)."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


# ----------------------------------------------------------------- forward + adjoint
def measure_adjoint(args, gpss, torch, flush, rank):
    """Forward render and path-replay adjoint of the differentiable workload
    (64^3 grids, 256x256, 64 spp): M path-vertices/s over recording forward + adjoint
    time and the ratio (t_recording_fwd + t_adj) / t_plain_fwd."""
    from paper_2603_00280_gb300 import workloads as W
    wl = W.differentiable(seed=12345 + 1000 * rank)
    cam, opts = wl["camera"], wl["opts"]
    S = gpss.Scene(wl["scene"])
    H, Wd = cam["height"], cam["width"]
    img = torch.empty((H, Wd, 3), device="cuda")
    g = torch.ones((H, Wd, 3), device="cuda")
    shape = wl["scene"]["objects"][0]["mean"].shape
    dm, dv = torch.zeros(shape, device="cuda"), torch.zeros(shape, device="cuda")
    da, dl = torch.zeros((1,) + shape, device="cuda"), torch.zeros(1, device="cuda")
    for _ in range(max(1, args.warmup)):
        gpss.render(S, cam, opts, image=img, stats=False, keep_path_radiance=True)
        gpss.render_adjoint(S, cam, opts, g, dm, dv, da, dl, stats=False)
    tp, tf, ta, verts, mism = [], [], [], 0, 0
    for _ in range(args.steps):
        flush.zero_()
        _, _, sp = gpss.render(S, cam, opts, image=img, stats=True)
        tp.append(sp["ms"])
        flush.zero_()
        _, _, st = gpss.render(S, cam, opts, image=img, stats=True, keep_path_radiance=True)
        tf.append(st["ms"])
        verts += st["vertices"]
        flush.zero_()
        sa = gpss.render_adjoint(S, cam, opts, g, dm, dv, da, dl, stats=True)
        ta.append(sa["ms"])
        mism += sa["aborted"]
    t_p, t_f, t_a = sum(tp), sum(tf), sum(ta)
    S.close()
    # inverse rendering from the perturbed start field toward the ground truth's image
    # (Adam through the forward render and the adjoint, L2 image loss)
    from paper_2603_00280_gb300 import optimize
    st = W.differentiable(start=True)
    fit = optimize.fit(st["scene"], img.clone(), cam, opts, steps=10)
    return {"workload": wl["name"], "image": [Wd, H], "spp": opts["spp"], "max_bounces": opts["max_bounces"],
            "value": verts / ((t_f + t_a) / 1e3) / 1e6, "unit": UNIT, "fwd_ms": t_p / args.steps,
            "fwd_recording_ms": t_f / args.steps, "adj_ms": t_a / args.steps,
            "ratio_fwd_plus_adj_over_fwd": (t_f + t_a) / t_p,
            "ratio_note": "(recording forward + adjoint) / plain forward render: the recording forward is the "
                          "adjoint's own kernel keeping each path's radiance, so the replay is bit-identical",
            "replay_mismatches": mism,
            "optimisation": {"ms_per_iteration": fit["ms_per_iteration"], "first_iteration_ms": fit["first_iteration_ms"],
                             "iterations": 10,
                             "loss_first": fit["losses"][0], "loss_last": fit["losses"][-1],
                             "step": "scene update + forward render (kept path radiance) + adjoint + Adam"}}


# ----------------------------------------------------------------- exact visible-normal sampling
def measure_vndf(args, gpss, torch, flush, wl, S, image):
    """The heterogeneous workload with the exact GPSS visible-normal sampler instead of
    the paper's mixture: throughput, and the summed per-pixel variance of the two
    estimators (same scene, same spp) -- the efficiency ratio is
    (var_mix t_mix) / (var_vndf t_vndf)."""
    import numpy as np
    cam = wl["camera"]
    res = {}
    for name, opts in (("mixture", wl["opts"]), ("vndf", dict(wl["opts"], sampler="vndf"))):
        for _ in range(2):
            gpss.render(S, cam, opts, image=image, stats=False)
        ms, verts = [], 0
        for _ in range(args.steps):
            flush.zero_()
            _, _, st = gpss.render(S, cam, opts, image=image, stats=True)
            ms.append(st["ms"])
            verts += st["vertices"]
        img, sq, _ = gpss.render(S, cam, opts, want_sqsum=True, stats=False)
        m = img.double().cpu().numpy()
        v = np.maximum(sq.double().cpu().numpy() / opts["spp"] - m * m, 0.0)
        res[name] = {"ms": sum(ms) / len(ms), "value": verts / (sum(ms) / 1e3) / 1e6, "var_sum": float(v.sum())}
    mix, vn = res["mixture"], res["vndf"]
    return {"workload": wl["name"], "unit": UNIT, "value_vndf": vn["value"], "value_mixture": mix["value"],
            "ms_vndf": vn["ms"], "ms_mixture": mix["ms"],
            "variance_ratio_vndf_over_mixture": vn["var_sum"] / mix["var_sum"],
            "efficiency_ratio": (mix["var_sum"] * mix["ms"]) / (vn["var_sum"] * vn["ms"]),
            "note": "per-pixel variance of one path's radiance summed over the image; same scene, spp and bounces"}


# ----------------------------------------------------------------- batched launch
def measure_batched(args, gpss, torch, flush):
    """The uneven 64-scene batch (images 64^2..512^2, grids 32^3..256^3, spp 4..64):
    one graph-replayed persistent launch with the autotuned shape against the 64
    separate gpss_render launches of the same jobs, queued back to back on the same
    stream.  Both trace the same paths (same indices, same random numbers; a rare
    decision may round differently in the two kernels), so their per-pixel errors are
    equal."""
    from paper_2603_00280_gb300 import workloads as W
    t0 = time.perf_counter()
    jobs = W.batched(args.batch_count, size_scale=args.batch_scale)
    gen_s = time.perf_counter() - t0
    scenes = [gpss.Scene(j["scene"]) for j in jobs]
    cams = [j["camera"] for j in jobs]
    opts = [j["opts"] for j in jobs]
    nodes = sum(o["mean"].size for j in jobs for o in j["scene"]["objects"])
    del jobs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = gpss.Batch(scenes, cams, opts, block_size=0)
    tune_s = time.perf_counter() - t0
    imgs = [torch.empty((c["height"], c["width"], 3), device="cuda") for c in cams]
    stream = torch.cuda.current_stream()

    def separate():
        for S, c, o, im in zip(scenes, cams, opts, imgs):
            gpss.render(S, c, o, image=im, stats=False)

    for _ in range(max(1, args.warmup)):
        B.render(images=imgs, stats=False)
        separate()
    torch.cuda.synchronize()
    g_ms, s_ms, verts, paths = [], [], 0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, st = B.render(images=imgs, stats=True)
        e1.record(stream)
        e1.synchronize()
        g_ms.append(e0.elapsed_time(e1))
        verts += st["vertices"]
        paths = st["paths"]
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        separate()
        e1.record(stream)
        e1.synchronize()
        s_ms.append(e0.elapsed_time(e1))
    cfg = B.config
    B.close()
    for S in scenes:
        S.close()
    tg, ts = sum(g_ms), sum(s_ms)
    return {"workload": "batched_%d_uneven" % args.batch_count, "scenes": args.batch_count,
            "size_scale": args.batch_scale, "paths_per_step": paths, "vertices_per_step": verts // args.steps,
            "grid_nodes": nodes, "graph_ms": tg / args.steps, "separate_ms": ts / args.steps,
            "speedup_graph_over_separate": ts / tg, "value_graph": verts / (tg / 1e3) / 1e6,
            "value_separate": verts / (ts / 1e3) / 1e6, "unit": UNIT, "launch": cfg,
            "autotune_s": tune_s, "generate_s": gen_s,
            "equal_error": "the same path indices and random numbers in both arms (the same estimator and per-pixel error)"}


# ----------------------------------------------------------------- arms
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.workload, image=args.image, spp=args.spp)
    vals = []
    desc = ""
    for i in range(args.warmup + args.steps):
        v, desc, cores, dt = oracle_sample(wl, max(2.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup))))
        if i >= args.warmup:
            vals.append((v, dt))
    value = statistics.median(v for v, _ in vals)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(d for _, d in vals),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_of(wl, "n/a (CPU)"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def time_renders(gpss, torch, S, cam, opts, image, flush, steps, warmup):
    """W warm-up renders, then K timed renders, each after an L2 flush: CUDA events on
    the launching stream around each step, and the render kernel's own event time."""
    for _ in range(warmup):
        gpss.render(S, cam, opts, image=image, stats=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    step_ms, kernel_ms, verts, ops, evals = [], [], 0, 0, 0
    stats = None
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, stats = gpss.render(S, cam, opts, image=image, stats=True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kernel_ms.append(stats["ms"])
        verts += stats["vertices"]
        ops += algorithmic_ops(stats)
        evals += evaluations(stats)
    return {"step_ms": step_ms, "kernel_ms": kernel_ms, "verts": verts, "ops": ops, "evals": evals, "stats": stats}


def work_of(stats, kernel_ms):
    return {"vertices_per_step": stats["vertices"], "null_collisions_per_step": stats["null_collisions"],
            "shadow_steps_per_step": stats["shadow_steps"], "paths_per_step": stats["paths"],
            "majorant_cells_per_step": stats["majorant_cells"], "max_path_events": stats.get("max_path_events"),
            "kernel_ms": statistics.mean(kernel_ms)}


def hbm_peak_gbs():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def measure_configs(args, gpss, torch, flush, rank, headline):
    """The other single-GPU configurations, each timed like the headline (fewer steps)."""
    out = {}
    for name in ("heterogeneous", "tiny_slab"):
        if name == headline:
            continue
        wl = workload(name, seed_offset=1000 * rank)
        S = gpss.Scene(wl["scene"])
        cam, opts = wl["camera"], wl["opts"]
        image = torch.empty((cam["height"], cam["width"], 3), device="cuda")
        t = time_renders(gpss, torch, S, cam, opts, image, flush, min(args.steps, 10), max(3, min(args.warmup, 3)))
        peak = peak_fp32_tops(torch)[0]
        achieved = t["ops"] / (sum(t["kernel_ms"]) / 1e3) / 1e12
        out[wl["name"]] = {"config": config_of(wl, "flushed between steps (256 MB write)"),
                           "value": t["verts"] / (sum(t["step_ms"]) / 1e3) / 1e6, "unit": UNIT,
                           "ms_per_step": statistics.mean(t["step_ms"]), "steps": len(t["step_ms"]),
                           "roofline_frac": achieved / peak, "achieved_tops": achieved,
                           "work": work_of(t["stats"], t["kernel_ms"])}
        S.close()
    return out


def run_ours(args):
    import numpy as np
    import torch
    from paper_2603_00280_gb300 import gpss

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    gpss.load()
    wl = workload(args.workload, seed_offset=1000 * rank, image=args.image, spp=args.spp)
    cam, opts = wl["camera"], wl["opts"]
    S = gpss.Scene(wl["scene"])
    H, W = cam["height"], cam["width"]
    image = torch.empty((H, W, 3), device="cuda", dtype=torch.float32)
    flush = torch.empty(64 * 1024 * 1024, device="cuda", dtype=torch.float32)  # 256 MB > L2
    for _ in range(args.warmup):
        gpss.render(S, cam, opts, image=image, stats=False)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t = time_renders(gpss, torch, S, cam, opts, image, flush, args.steps, 0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    stats, kernel_ms = t["stats"], t["kernel_ms"]
    total_ms, all_verts = job_totals(sum(t["step_ms"]), t["verts"], dist, "cuda")
    value = all_verts / (total_ms / 1e3) / 1e6

    # e2e through the C-ABI with host buffers: upload the grids from pinned host
    # memory (scene update + majorant rebuild) and read the image back, every step
    e2e = None
    if not args.no_e2e:
        objs = []
        h2d = 0
        for o in wl["scene"]["objects"]:
            d = {k: o[k] for k in ("bbox_min", "bbox_max", "length_scale")}
            for k in ("mean", "var", "albedo"):
                d[k] = torch.from_numpy(np.ascontiguousarray(o[k])).pin_memory()
                h2d += d[k].numel() * 4
            objs.append(d)
        host_img = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
        e2e_ms, e2e_verts = [], 0
        e_warm, e_steps = min(args.warmup, 3), min(args.steps, 10)
        for i in range(e_warm + e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            S.update(objs)
            _, _, st = gpss.render(S, cam, opts, image=host_img.numpy(), stats=True)
            t1 = time.perf_counter()
            if i >= e_warm:
                e2e_ms.append(1e3 * (t1 - t0))
                e2e_verts += st["vertices"]
        e_ms, e_verts = job_totals(sum(e2e_ms), e2e_verts, dist, "cuda")
        e2e = {"value": e_verts / (e_ms / 1e3) / 1e6, "unit": UNIT, "steps": e_steps,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": H * W * 3 * 4}
        del objs
    S.close()

    configs = None if (args.no_configs or world > 1) else measure_configs(args, gpss, torch, flush, rank, args.workload)
    adj = None if args.no_adjoint else measure_adjoint(args, gpss, torch, flush, rank)
    batched = None if (args.no_batched or world > 1) else measure_batched(args, gpss, torch, flush)
    vndf = None
    if not (args.no_vndf or world > 1):
        wv = workload("heterogeneous", seed_offset=1000 * rank)
        Sv = gpss.Scene(wv["scene"])
        img_v = torch.empty((wv["camera"]["height"], wv["camera"]["width"], 3), device="cuda")
        vndf = measure_vndf(args, gpss, torch, flush, wv, Sv, img_v)
        Sv.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    per_eval, per_vertex, bytes_eval = opcounts()
    peak, sms, mhz, peak_src = peak_fp32_tops(torch)
    kernel_s = sum(kernel_ms) / 1e3
    achieved = t["ops"] / kernel_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": measured_traffic(wl["name"]),
            "note": "FP32 issue roofline: %d SMs x 128 lanes x %.0f MHz (%s), one FMA = one op; algorithmic ops = "
                    "%d per extinction evaluation + %d per vertex (paper_2603_00280_gb300/opcounts.json, tallied "
                    "from the formulas)" % (sms, mhz, peak_src, per_eval, per_vertex)}
    hbm, hbm_src = hbm_peak_gbs()
    gbs = t["evals"] * bytes_eval / kernel_s / 1e9
    roof_hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "note": "algorithmic field gathers: %d B (8 corners x (mean, variance)) per extinction evaluation; "
                        "peak %s" % (bytes_eval, hbm_src)}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": config_of(wl, "inputs larger than L2 and L2 flushed between steps (256 MB write)"),
           "roofline": roof, "roofline_hbm": roof_hbm, "e2e": e2e, "gpu_launches": args.steps,
           "clocks": clk, "configs": configs, "fwd_adjoint": adj, "batched": batched, "exact_vndf": vndf,
           "work": work_of(stats, kernel_ms)}
    if world == 1 and not args.no_cpu_baseline:
        v, desc, cores, _ = oracle_sample(wl, args.cpu_seconds)
        v1, desc1, _, _ = oracle_sample(wl, max(2.0, args.cpu_seconds / 2), threads=1)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                               "one_core": {"value": v1, "unit": UNIT, "cores": 1, "sample": desc1}}
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
