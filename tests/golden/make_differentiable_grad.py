"""Writes tests/golden/differentiable_grad.json: the FP64 oracle's adjoint on the
differentiable configuration at full size, the reference of the GPU adjoint's
per-voxel test (tests/test_gpu_adjoint_voxels.py).

Configuration: the start field of the differentiable workload (64^3 mean,
variance and albedo grids, l = 0.012; 256x256 perspective camera, procedural sky,
32 bounces).  The oracle samples phase functions exactly (its visible-normal
sampler: the same expected gradient as the paper's mixture, which the GPU side
runs, with bounded path weights, so batch standard errors are reliable).  Loss: the sum of all three
channels over a 16x16 window of the image (d_image = 1 there, 0 elsewhere).
Voxels: 32 nodes (seed 3) drawn from the shell nodes (|mu| < 3 sigma, reading Q18)
that project into the window's interior and that the camera sees (oracle
transmittance from the eye above 0.05).

The oracle (orc_render_grad: path replay of its regular-tracking estimator,
partials from dual numbers) runs K independent batches (seeds 1..K); the file
stores each gradient's batch mean and standard error.  Only ``oracle/`` computes
anything here; the workload generator supplies the inputs.

    python tests/golden/make_differentiable_grad.py [--batches K] [--spp S] [--threads T]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2603_00280_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "differentiable_grad.json")
WINDOW = (100, 116, 120, 136)  # rows r0:r1, cols c0:c1


def project(cam, p):
    """Pixel coordinates of points p under the perspective camera (the camera model of
    orc_camera_ray inverted: forward f, right f x up, image up right x f)."""
    eye, la, up = (np.asarray(cam[k], np.float64) for k in ("eye", "look_at", "up"))
    f = la - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(math.radians(cam["fov_y_deg"]) / 2)
    asp = cam["width"] / cam["height"]
    v = p - eye
    vf = v @ f
    px = ((v @ r) / vf / (th * asp) + 1) / 2 * cam["width"]
    py = (1 - (v @ u) / vf / th) / 2 * cam["height"]
    return px, py


def select_voxels(wl, S, count=32, seed=3):
    cam = wl["camera"]
    obj = wl["scene"]["objects"][0]
    n = obj["mean"].shape[0]
    p = W.node_coords(obj["bbox_min"], obj["bbox_max"], (n, n, n)).reshape(-1, 3)
    mean = np.asarray(obj["mean"], np.float64).reshape(-1)
    sig = np.sqrt(np.asarray(obj["var"], np.float64)).reshape(-1)
    px, py = project(cam, p)
    r0, r1, c0, c1 = WINDOW
    cand = np.flatnonzero((np.abs(mean) < 3 * sig) & (py >= r0 + 2) & (py < r1 - 2) & (px >= c0 + 2) & (px < c1 - 2))
    eye = np.asarray(cam["eye"], np.float64)
    vis = []
    for i in cand:
        dvec = p[i] - eye
        dist = float(np.linalg.norm(dvec))
        if oracle.transmittance(S, eye, dvec / dist, dist) > 0.05:
            vis.append(i)
    vis = np.array(vis)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(vis, count, replace=False)), len(cand), len(vis)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batches", type=int, default=16)
    ap.add_argument("--spp", type=int, default=256, help="samples per pixel per batch (voxel gradients)")
    ap.add_argument("--l-batches", type=int, default=8)
    ap.add_argument("--l-spp", type=int, default=16, help="samples per pixel per batch (length-scale gradient)")
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    wl = W.differentiable(start=True)
    sc, cam, opts = wl["scene"], wl["camera"], wl["opts"]
    S = oracle.Scene(sc)
    nodes, n_cand, n_vis = select_voxels(wl, S)
    r0, r1, c0, c1 = WINDOW
    g = np.zeros((cam["height"], cam["width"], 3))
    g[r0:r1, c0:c1, :] = 1.0
    win = dict(rows=(r0, r1, 1), cols=(c0, c1), threads=a.threads)
    t0 = time.time()
    rows, paths = [], 0
    for b in range(a.batches):
        (r,), st = oracle.render_grad(S, cam, dict(opts, spp=a.spp, seed=1 + b, sampler="vndf"), g, nodes=[nodes],
                                      want=("mean", "var", "albedo"), **win)
        assert st["mismatch"] == 0
        paths += st["paths"]
        rows.append(np.concatenate([r["mean"], r["var"], r["albedo"][0]]))
        print("batch %d/%d  %.0f s" % (b + 1, a.batches, time.time() - t0), flush=True)
    e = np.array(rows)
    m, se = e.mean(0), e.std(0, ddof=1) / math.sqrt(len(e))
    lrows = []
    for b in range(a.l_batches):
        (r,), st = oracle.render_grad(S, cam, dict(opts, spp=a.l_spp, seed=1001 + b, sampler="vndf"), g,
                                      nodes=[nodes[:1]], want=("l",), **win)
        paths += st["paths"]
        lrows.append(r["l"])
        print("l batch %d/%d  %.0f s" % (b + 1, a.l_batches, time.time() - t0), flush=True)
    lm, lse = float(np.mean(lrows)), float(np.std(lrows, ddof=1) / math.sqrt(len(lrows)))
    k = len(nodes)
    out = {
        "generated_by": "tests/golden/make_differentiable_grad.py (FP64 oracle, orc_render_grad)",
        "workload": "differentiable_64 start field (64^3; 256x256 perspective, sky, 32 bounces); oracle sampler: "
                    "exact visible normals",
        "loss": "sum of all channels of the image over the window (d_image = 1 there, 0 elsewhere)",
        "window": list(WINDOW),
        "voxel_rule": "32 nodes (seed 3) among shell nodes |mu| < 3 sigma projecting into the window interior "
                      "with oracle transmittance from the eye > 0.05",
        "candidates": int(n_cand), "visible": int(n_vis),
        "nodes": [int(v) for v in nodes],
        "batches": a.batches, "spp_per_batch": a.spp, "seeds": list(range(1, 1 + a.batches)),
        "l_batches": a.l_batches, "l_spp_per_batch": a.l_spp,
        "paths": int(paths), "seconds": round(time.time() - t0, 1),
        "d_mean": {"mean": m[:k].tolist(), "se": se[:k].tolist()},
        "d_variance": {"mean": m[k:2 * k].tolist(), "se": se[k:2 * k].tolist()},
        "d_albedo": {"mean": m[2 * k:].tolist(), "se": se[2 * k:].tolist()},
        "d_length_scale": {"mean": lm, "se": lse},
    }
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", OUT, "in %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
