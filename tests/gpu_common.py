"""Shared helpers of the GPU parity tests (no method arithmetic)."""
import math

import numpy as np

from paper_2603_00280_gb300 import workloads as W

REL = 1e-5  # deterministic parity bar (relative), from the spec requirement


def dyadic_hetero(n_log2=5, length_scale=0.01, sigma_lo=0.01, sigma_hi=0.1, seed=0, channels=1):
    """Heterogeneous sphere-noise scene on a grid with 2^k + 1 nodes over [-0.5, 0.5]^3,
    so that h = 2^-k and cell coordinates of dyadic positions are exact in FP32."""
    n = (1 << n_log2) + 1
    bmin, bmax = (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5)
    p = W.node_coords(bmin, bmax, (n, n, n))
    mean = W.sdf_sphere(p, (0.0, 0.0, 0.0), 0.3) + 0.02 * W.value_noise(p, seed)
    var = sigma_lo ** 2 + (sigma_hi ** 2 - sigma_lo ** 2) * (p[..., 0] + 0.5)
    if channels == 3:
        alb = np.random.default_rng(seed + 7).uniform(0.3, 0.95, size=(3, n, n, n)).astype(np.float32)
    else:
        alb = 0.8
    obj = W.make_object(mean, var, alb, bmin, bmax, length_scale)
    return {"objects": [obj], "light": W.sky_light()}


def dyadic_points(n, seed, lo=-0.45, hi=0.45):
    """Positions that are multiples of 2^-24 (exact in FP32, exact offsets from -0.5)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, size=(n, 3))
    return (np.round(x * 2 ** 24) / 2 ** 24).astype(np.float32)


def unit_dirs(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32)


def rel_err(a, b, floor=0.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


# The GPU film accumulates per-pixel sums with FP32 atomics.  For a nearly
# deterministic pixel (sky seen through jittered rays) every addition rounds the
# same way, so the sum of n equal terms can drift by up to n half-ulps of the
# running sum: a relative error of n 2^-25, which the sample variance (nearly 0
# there) does not show.  The GPU standard error is floored at that bound (plus a
# tiny constant for 0-valued pixels).
def film_floor(mean, spp):
    return np.abs(mean) * spp * 2.0 ** -25 + 1e-9


def robust_var(v):
    """Per-sample variance map (H, W, 3) of one side, made robust to its own small
    samples: the larger of the pixel's estimate and the mean of its 3x3 neighbourhood
    (edges clamped).  The variance varies slowly across an image except at
    silhouettes, where a pixel's few samples may all miss (or all hit) the object and
    its own estimate collapses; the neighbourhood there includes both."""
    v = np.asarray(v, np.float64)
    if v.ndim != 3 or v.shape[0] < 2 or v.shape[1] < 2:
        return v
    p = np.pad(v, ((1, 1), (1, 1), (0, 0)), mode="edge")
    H, W = v.shape[:2]
    nb = sum(p[i:i + H, j:j + W] for i in range(3) for j in range(3)) / 9.0
    return np.maximum(v, nb)


def image_z(gpu_mean, gpu_sqsum, gpu_spp, orc_sum, orc_sumsq, orc_spp):
    """Per-pixel z of the difference between two independent Monte Carlo images, each
    with the standard error of its own samples only (nothing is pooled between the
    two sides): per-sample variances from each side's own sums of squares, made
    robust by robust_var, over that side's sample count.  The oracle renders with its
    exact visible-normal sampler where the object allows it (bounded path weights);
    the GPU takes many more samples than the oracle."""
    gm = np.asarray(gpu_mean, np.float64)
    gv = robust_var(np.maximum(np.asarray(gpu_sqsum, np.float64) / gpu_spp - gm ** 2, 0.0)) / gpu_spp
    gv = np.maximum(gv, film_floor(gm, gpu_spp) ** 2)
    om = np.asarray(orc_sum, np.float64) / orc_spp
    ov = robust_var(np.maximum(np.asarray(orc_sumsq, np.float64) / orc_spp - om ** 2, 0.0)) / orc_spp
    se = np.sqrt(gv + ov)
    z = np.where(se > 0, (gm - om) / np.where(se > 0, se, 1.0), np.where(np.abs(gm - om) > 1e-6, np.inf, 0.0))
    return z, gm, om, np.sqrt(gv), np.sqrt(ov)


def check_image_parity(gm, gse, om, ose, frac3=0.01):
    """The image parity bar: at most 1% of the compared pixel-channels with |z| > 3
    (0.27% expected; at least one such entry is allowed when fewer than 100 are
    compared, where 1% is not a whole entry), every channel's image total within 3
    standard errors, and no entry beyond |z| = 6.  Returns (ok, a one-line report
    with the worst entries)."""
    se = np.sqrt(gse ** 2 + ose ** 2)
    z = np.where(se > 0, (gm - om) / np.where(se > 0, se, 1), 0.0)
    n = z.size
    n3 = int(np.sum(np.abs(z) > 3))
    allowed = max(1, int(frac3 * n))
    ch = gm.reshape(-1, gm.shape[-1])
    tz = (ch.sum(0) - om.reshape(ch.shape).sum(0)) / np.sqrt(
        (gse.reshape(ch.shape) ** 2).sum(0) + (ose.reshape(ch.shape) ** 2).sum(0) + 1e-300)
    worst = np.argsort(-np.abs(z).reshape(-1))[:6]
    fl = lambda a: a.reshape(-1)
    report = "n=%d |z|>3: %d (allowed %d) max|z|=%.2f total z=%s worst (idx, z, gpu, oracle, gse, ose): %s" % (
        n, n3, allowed, float(np.abs(z).max()), np.round(tz, 2).tolist(),
        [(int(i), round(float(fl(z)[i]), 2), float("%.4g" % fl(gm)[i]), float("%.4g" % fl(om)[i]),
          float("%.3g" % fl(gse)[i]), float("%.3g" % fl(ose)[i])) for i in worst])
    ok = n3 <= allowed and bool(np.all(np.abs(tz) < 3)) and float(np.abs(z).max()) < 6
    return ok, report


def two_spheres_rgb():
    """Two overlapping GPSS spheres on their own dyadic grids, RGB albedo: the
    extinctions add and the scattering object is chosen by extinction."""
    objs = []
    rng = np.random.default_rng(4)
    for c, r, v, lo, hi in [((-0.1, 0, 0), 0.25, 4e-3, (-0.5, -0.375, -0.375), (0.25, 0.375, 0.375)),
                            ((0.15, 0.05, 0), 0.2, 1e-2, (-0.125, -0.25, -0.25), (0.5, 0.375, 0.375))]:
        n = (int(round((hi[0] - lo[0]) * 32)) + 1, int(round((hi[1] - lo[1]) * 32)) + 1, int(round((hi[2] - lo[2]) * 32)) + 1)
        p = W.node_coords(lo, hi, n)
        alb = rng.uniform(0.3, 0.95, size=(3, n[2], n[1], n[0])).astype(np.float32)
        objs.append(W.make_object(W.sdf_sphere(p, c, r), v, alb, lo, hi, 0.05))
    return {"objects": objs, "light": W.sky_light()}
