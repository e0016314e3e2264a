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


# The GPU film accumulates per-pixel sums with FP32 atomics; its variance estimate
# E[L^2] - mean^2 cancels for nearly deterministic pixels (e.g. sky seen through
# jittered rays).  A floor of FILM_REL * |mean| on the GPU standard error covers
# the FP32 accumulation error of sums of up to ~10^4 samples.
FILM_REL = 2e-5


def image_z(gpu_mean, gpu_sqsum, gpu_spp, orc_sum, orc_sumsq, orc_spp, orc_sample_var=None):
    """Per-pixel z of the difference between two Monte Carlo images.  orc_sample_var:
    the per-sample variance of the oracle's estimator measured by a larger run of the
    same estimator (the GPU with the oracle's sampler); it raises the oracle's own
    small-sample estimate where that missed the heavy tail."""
    gm = np.asarray(gpu_mean, np.float64)
    gv = np.maximum(np.asarray(gpu_sqsum, np.float64) / gpu_spp - gm ** 2, 0.0) / gpu_spp
    gv = np.maximum(gv, (FILM_REL * np.abs(gm)) ** 2)
    om = orc_sum / orc_spp
    ovar = np.maximum(orc_sumsq / orc_spp - om ** 2, 0.0)
    if orc_sample_var is not None:
        ovar = np.maximum(ovar, orc_sample_var)
    # Where both sides sample the same per-pixel distribution (the same sampler), the
    # path weights are heavy tailed, so the smaller sample's variance estimate is
    # raised to the pooled estimate (dominated by the larger, GPU sample).
    pooled = (gv * gpu_spp * gpu_spp + ovar * orc_spp) / (gpu_spp + orc_spp)
    ov = np.maximum(ovar, pooled) / orc_spp
    se = np.sqrt(gv + ov)
    z = np.where(se > 0, (gm - om) / np.where(se > 0, se, 1.0), np.where(np.abs(gm - om) > 1e-6, np.inf, 0.0))
    return z, gm, om, np.sqrt(gv), np.sqrt(ov)


def check_image_parity(gm, gse, om, ose, frac4=0.01, block=4):
    """Heavy-tail-robust parity criteria for two Monte Carlo images:
    - at most `frac4` of the pixels with |z| > 4 (the mixture sampler's path
      weights are heavy tailed, so per-pixel sample errors underestimate now and
      then; |z| > 3 is reported, not asserted);
    - block means over `block` x `block` pixels: at most 3% with |z| > 3;
    - the image total within 4 standard errors."""
    se = np.sqrt(gse ** 2 + ose ** 2)
    z = np.where(se > 0, (gm - om) / np.where(se > 0, se, 1), 0.0)
    out = {"frac_z3": float(np.mean(np.abs(z) > 3)), "frac_z4": float(np.mean(np.abs(z) > 4))}
    H, W = gm.shape[:2]
    hb, wb = H // block * block, W // block * block
    if hb and wb:
        def blk(a, sq=False):
            a = a[:hb, :wb].reshape(hb // block, block, wb // block, block, -1)
            return (a ** 2).sum(axis=(1, 3)) if sq else a.sum(axis=(1, 3))
        bz = (blk(gm) - blk(om)) / np.sqrt(blk(gse, True) + blk(ose, True) + 1e-300)
        out["block_frac_z3"] = float(np.mean(np.abs(bz) > 3))
    else:
        out["block_frac_z3"] = 0.0
    out["total_z"] = float((gm.sum() - om.sum()) / np.sqrt(np.sum(gse ** 2) + np.sum(ose ** 2)))
    ok = out["frac_z4"] <= frac4 and out["block_frac_z3"] <= 0.03 and abs(out["total_z"]) < 4
    return ok, out


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


def sample_var(mean, sqsum, spp):
    """Per-sample variance of a GPU image from its sum of squares."""
    m = np.asarray(mean, np.float64)
    return np.maximum(np.asarray(sqsum, np.float64) / spp - m * m, 0.0)
