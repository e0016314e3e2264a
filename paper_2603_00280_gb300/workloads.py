"""Seeded synthetic inputs for the GPSS renderer (scenes, cameras, lights, options).

This module is the one place both sides of every parity check take their
inputs from: the CUDA library and the CPU oracle read the same float32 grids.
It holds geometry (signed distances), seeded value noise and parameter ramps
only -- none of the renderer's arithmetic.

The paper's own scenes (meshes, reference renders) are not available, so these
workloads stand in for them with the paper's parameter regimes: surface-like
shells with sigma = 0.01 and roughness 0.1..1 (Sec. 5.1), strongly anisotropic
and isotropic kernels, and spatially varying variance (Sec. 5.2).

Every workload is a dict ``{"name", "scene", "camera", "opts"}``:

- ``scene = {"objects": [obj, ...], "light": light}`` with
  ``obj = {"mean", "var": float32 (nz, ny, nx), "albedo": float32 (C, nz, ny, nx),
  "bbox_min", "bbox_max": (3,), "length_scale": float}`` (node-centred grids
  spanning the box, x fastest) and
  ``light = {"type": "directional" | "sky" | "uniform", "dir": (3,), "radiance": (3,)}``;
- ``camera = {"type": "ortho" | "perspective", "eye", "look_at", "up",
  "fov_y_deg", "ortho_w", "ortho_h", "width", "height"}``;
- ``opts = {"spp", "max_bounces", "seed", "mix_R"}``.
"""
from __future__ import annotations

import math

import numpy as np

# ------------------------------------------------------------------ noise

_NOISE_LO = -1.5  # lattice origin (world units); covers every scene box used here


def value_noise(points: np.ndarray, seed: int, freqs=(8, 16, 32), amps=(1.0, 0.5, 0.25)) -> np.ndarray:
    """Three-octave value noise in [-1, 1] at ``points`` (..., 3).

    Lattice values are 2u-1 with u from numpy's PCG64 seeded by (seed, octave);
    interpolation is trilinear with smoothstep weights 3w^2-2w^3; the octave sum
    is divided by the sum of the amplitudes.
    """
    p = np.asarray(points, dtype=np.float64)
    out = np.zeros(p.shape[:-1])
    for octave, (f, a) in enumerate(zip(freqs, amps)):
        n, lat = _lattice(seed, octave, f)
        g = (p - _NOISE_LO) * f
        i = np.clip(np.floor(g).astype(np.int64), 0, n - 2)
        w = np.clip(g - i, 0.0, 1.0)
        w = w * w * (3.0 - 2.0 * w)
        acc = np.zeros(p.shape[:-1])
        for c in range(8):
            cx, cy, cz = c & 1, (c >> 1) & 1, (c >> 2) & 1
            wt = ((w[..., 0] if cx else 1 - w[..., 0]) * (w[..., 1] if cy else 1 - w[..., 1])
                  * (w[..., 2] if cz else 1 - w[..., 2]))
            acc += wt * lat[i[..., 0] + cx, i[..., 1] + cy, i[..., 2] + cz]
        out += a * acc
    return out / float(sum(amps))


def _lattice(seed: int, octave: int, f: float):
    n = int(math.ceil(3.0 * f)) + 3
    return n, 2.0 * np.random.default_rng([seed, octave]).random((n, n, n)) - 1.0


def value_noise_grid(bmin, bmax, n, seed: int, freqs=(8, 16, 32), amps=(1.0, 0.5, 0.25)) -> np.ndarray:
    """``value_noise`` at the nodes of a node-centred grid (``node_coords``), shape
    (nz, ny, nx).  The interpolation weights factor per axis, so each octave is
    three one-dimensional interpolations of the lattice (x, then y, then z) instead
    of eight corner lookups per node; the values equal ``value_noise`` up to the
    order of the floating-point additions."""
    axes = [np.linspace(bmin[a], bmax[a], n[a]) for a in range(3)]
    out = np.zeros((n[2], n[1], n[0]))
    for octave, (f, a) in enumerate(zip(freqs, amps)):
        m, lat = _lattice(seed, octave, f)
        idx, wts = [], []
        for c in axes:
            g = (c - _NOISE_LO) * f
            i = np.clip(np.floor(g).astype(np.int64), 0, m - 2)
            w = np.clip(g - i, 0.0, 1.0)
            idx.append(i)
            wts.append(w * w * (3.0 - 2.0 * w))
        (ix, iy, iz), (wx, wy, wz) = idx, wts
        A = (1 - wx)[:, None, None] * lat[ix] + wx[:, None, None] * lat[ix + 1]                    # (nx, m, m)
        B = (1 - wy)[None, :, None] * A[:, iy, :] + wy[None, :, None] * A[:, iy + 1, :]            # (nx, ny, m)
        C = (1 - wz)[None, None, :] * B[:, :, iz] + wz[None, None, :] * B[:, :, iz + 1]            # (nx, ny, nz)
        out += a * C.transpose(2, 1, 0)
    return out / float(sum(amps))


# ------------------------------------------------------------------ geometry

def node_coords(bmin, bmax, n):
    """World coordinates (nz, ny, nx, 3) of a node-centred grid with n = (nx, ny, nz) nodes."""
    xs = [np.linspace(bmin[a], bmax[a], n[a]) for a in range(3)]
    z, y, x = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return np.stack([x, y, z], axis=-1)


def sdf_sphere(p, center, r):
    return np.linalg.norm(p - np.asarray(center), axis=-1) - r


def sdf_box(p, center, half):
    q = np.abs(p - np.asarray(center)) - np.asarray(half)
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(np.max(q, axis=-1), 0.0)
    return outside + inside


def sdf_torus_z(p, center, R, r):
    q = p - np.asarray(center)
    ring = np.sqrt(q[..., 0] ** 2 + q[..., 1] ** 2) - R
    return np.sqrt(ring ** 2 + q[..., 2] ** 2) - r


def make_object(mean, var, albedo, bmin, bmax, length_scale):
    mean = np.ascontiguousarray(mean, dtype=np.float32)
    var = np.ascontiguousarray(np.broadcast_to(var, mean.shape), dtype=np.float32)
    albedo = np.asarray(albedo, dtype=np.float32)
    if albedo.ndim == 0:
        albedo = np.full((1,) + mean.shape, float(albedo), dtype=np.float32)
    elif albedo.ndim == 3:
        albedo = albedo[None]
    return {"mean": mean, "var": var, "albedo": np.ascontiguousarray(albedo),
            "bbox_min": np.asarray(bmin, dtype=np.float64), "bbox_max": np.asarray(bmax, dtype=np.float64),
            "length_scale": float(length_scale)}


def sky_light(scale=1.0):
    return {"type": "sky", "dir": (0.0, 0.0, 1.0), "radiance": (scale, scale, scale)}


def uniform_light(value=1.0):
    return {"type": "uniform", "dir": (0.0, 0.0, 1.0), "radiance": (value, value, value)}


def directional_light(direction=(0.0, 0.0, 1.0), irradiance=1.0):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return {"type": "directional", "dir": tuple(d), "radiance": (irradiance,) * 3}


def perspective_camera(width, height, eye=(0.0, -1.8, 0.9), look_at=(0.0, 0.0, 0.0), fov_y_deg=40.0):
    return {"type": "perspective", "eye": tuple(eye), "look_at": tuple(look_at), "up": (0.0, 0.0, 1.0),
            "fov_y_deg": float(fov_y_deg), "ortho_w": 1.0, "ortho_h": 1.0, "width": int(width), "height": int(height)}


def ortho_camera_45(width, height, film=1.2):
    """Orthographic camera looking along d = (cos 45, 0, -sin 45) at the origin."""
    d = np.array([math.cos(math.pi / 4), 0.0, -math.sin(math.pi / 4)])
    eye = -2.0 * d
    return {"type": "ortho", "eye": tuple(eye), "look_at": (0.0, 0.0, 0.0), "up": (0.0, 0.0, 1.0),
            "fov_y_deg": 40.0, "ortho_w": float(film), "ortho_h": float(film), "width": int(width), "height": int(height)}


# ------------------------------------------------------------------ workloads

def tiny_slab(width=64, height=64, spp=16, max_bounces=8, seed=0, nodes=(33, 33, 9), sigma=0.05,
              length_scale=0.02, albedo=0.8, light=None):
    """Plain method, tiny: a GPSS slab whose mean is the signed distance to z=0.

    Box [-0.5,0.5]^2 x [-0.1,0.1]; mean = z (reproduced exactly by trilinear
    interpolation); constant variance sigma^2; SE length scale l; orthographic
    camera at 45 degrees; one directional light straight down onto the slab.
    """
    bmin, bmax = (-0.5, -0.5, -0.1), (0.5, 0.5, 0.1)
    p = node_coords(bmin, bmax, nodes)
    obj = make_object(p[..., 2], sigma * sigma, albedo, bmin, bmax, length_scale)
    return {"name": "tiny_slab",
            "scene": {"objects": [obj], "light": light or directional_light((0.0, 0.0, 1.0), 1.0)},
            "camera": ortho_camera_45(width, height),
            "opts": {"spp": spp, "max_bounces": max_bounces, "seed": seed, "mix_R": 0.5}}


def heterogeneous(n=128, width=512, height=512, spp=64, max_bounces=32, seed=0, noise_seed=0,
                  length_scale=0.01, albedo=0.8):
    """Heterogeneous GPSS: sphere of radius 0.3 plus 0.02 of seeded value noise
    on an n^3 grid over [-0.5,0.5]^3; variance ramps from 1e-4 to 1e-2 along x;
    perspective camera, procedural sky."""
    bmin, bmax = (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5)
    p = node_coords(bmin, bmax, (n, n, n))
    mean = sdf_sphere(p, (0.0, 0.0, 0.0), 0.3) + 0.02 * value_noise_grid(bmin, bmax, (n, n, n), noise_seed)
    var = 1e-4 + (0.01 - 1e-4) * (p[..., 0] + 0.5)
    obj = make_object(mean, var, albedo, bmin, bmax, length_scale)
    return {"name": "heterogeneous_%d" % n,
            "scene": {"objects": [obj], "light": sky_light()},
            "camera": perspective_camera(width, height),
            "opts": {"spp": spp, "max_bounces": max_bounces, "seed": seed, "mix_R": 0.5}}


def surface_to_volume(n=256, width=1024, height=1024, spp=256, max_bounces=64, seed=0):
    """Three objects (torus, box, sphere) on their own n^3 grids, variances
    1e-6 (surface-like), 2.24e-4 and 0.05 (volume-like); RGB albedo per node
    drawn from U[0.3, 0.95] (seed 7)."""
    rng = np.random.default_rng(7)
    specs = [("torus", (-0.55, 0.0, 0.0), 1e-6), ("box", (0.0, 0.0, 0.0), 2.24e-4), ("sphere", (0.55, 0.0, 0.0), 0.05)]
    objs = []
    for kind, c, v in specs:
        pad = min(3.0 * math.sqrt(v), 0.25)
        if kind == "torus":
            half = np.array([0.33, 0.33, 0.08])
        elif kind == "box":
            half = np.array([0.2, 0.2, 0.2])
        else:
            half = np.array([0.25, 0.25, 0.25])
        bmin = np.asarray(c) - half - pad
        bmax = np.asarray(c) + half + pad
        p = node_coords(bmin, bmax, (n, n, n))
        if kind == "torus":
            mean = sdf_torus_z(p, c, 0.25, 0.08)
        elif kind == "box":
            mean = sdf_box(p, c, (0.2, 0.2, 0.2))
        else:
            mean = sdf_sphere(p, c, 0.25)
        alb = rng.uniform(0.3, 0.95, size=(3, n, n, n)).astype(np.float32)
        objs.append(make_object(mean, v, alb, bmin, bmax, 0.01))
    return {"name": "surface_to_volume_%d" % n,
            "scene": {"objects": objs, "light": sky_light()},
            "camera": perspective_camera(width, height, eye=(0.0, -2.6, 1.2)),
            "opts": {"spp": spp, "max_bounces": max_bounces, "seed": seed, "mix_R": 0.5}}


def differentiable(n=64, width=256, height=256, spp=64, max_bounces=32, seed=12345, start=False):
    """Differentiable-render workload: ground truth = sphere-noise field (noise
    seed 1), variance ramp, albedo 0.8, l = 0.01.  ``start=True`` returns the
    perturbed starting point (mean + 0.01 noise(seed 2), variance x2, albedo
    0.6, l = 0.012)."""
    bmin, bmax = (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5)
    p = node_coords(bmin, bmax, (n, n, n))
    mean = sdf_sphere(p, (0.0, 0.0, 0.0), 0.3) + 0.02 * value_noise_grid(bmin, bmax, (n, n, n), 1)
    var = 1e-4 + (0.01 - 1e-4) * (p[..., 0] + 0.5)
    albedo, l = 0.8, 0.01
    if start:
        mean = mean + 0.01 * value_noise_grid(bmin, bmax, (n, n, n), 2)
        var = 2.0 * var
        albedo, l = 0.6, 0.012
    obj = make_object(mean, var, albedo, bmin, bmax, l)
    return {"name": "differentiable_%d" % n,
            "scene": {"objects": [obj], "light": sky_light()},
            "camera": perspective_camera(width, height),
            "opts": {"spp": spp, "max_bounces": max_bounces, "seed": seed, "mix_R": 0.5}}


def tangent_swirl(p, twist=0.25):
    """Tangent field (3, nz, ny, nx) swirling about z: t = (-y, x, twist) at the node
    coordinates p (nz, ny, nx, 3)."""
    return np.ascontiguousarray(np.stack([-p[..., 1], p[..., 0], np.full(p.shape[:-1], twist)]), dtype=np.float32)


def correlation_ramp(p, lo=0.5, hi=1.5, axis=2):
    """Correlation-scale factors rising linearly from lo to hi along `axis` over
    [-0.5, 0.5] (the correlation grows from bottom to top, as in the paper's
    non-stationary sweeps)."""
    return np.ascontiguousarray(lo + (hi - lo) * (p[..., axis] + 0.5), dtype=np.float32)


def with_kernel(obj, l_b_ratio=2.0, l_n_ratio=0.5, tangent=True, correlation=True):
    """Returns a copy of an object on a node grid with an anisotropic (l_b = l_b_ratio
    l_t along the swirl's bitangent, l_n = l_n_ratio l_t) and non-stationary
    (correlation ramp) kernel."""
    o = dict(obj)
    nz, ny, nx = obj["mean"].shape
    p = node_coords(obj["bbox_min"], obj["bbox_max"], (nx, ny, nz))
    l = obj["length_scale"]
    if tangent:
        o["tangent"] = tangent_swirl(p)
        o["length_scale_b"] = l * l_b_ratio
    if l_n_ratio != 1.0:
        o["length_scale_n"] = l * l_n_ratio
    if correlation:
        o["correlation_scale"] = correlation_ramp(p)
    return o


def nonstationary(n=64, width=256, height=256, spp=64, max_bounces=32, seed=0, length_scale=0.02,
                  l_b_ratio=2.0, l_n_ratio=0.5):
    """The heterogeneous sphere-noise GPSS (variance ramp 1e-4..1e-2 along x) with an
    anisotropic, non-stationary kernel: l_t = length_scale, l_b = l_b_ratio l_t along
    the bitangent of a tangent field swirling about z, l_n = l_n_ratio l_t, every l
    scaled by a factor rising from 0.5 at the bottom to 1.5 at the top."""
    wl = heterogeneous(n=n, width=width, height=height, spp=spp, max_bounces=max_bounces, seed=seed,
                       length_scale=length_scale)
    wl["scene"]["objects"] = [with_kernel(wl["scene"]["objects"][0], l_b_ratio, l_n_ratio)]
    wl["name"] = "nonstationary_%d" % n
    return wl


def batched_scene(s: int, size_scale: float = 1.0):
    """Scene s (0..63) of the batched workload: image side 64..512, grid 32..256
    nodes per axis, spp 4..64, a sphere / plane / box mean with 0.02 noise and a
    constant variance log-uniform in [1e-6, 0.05]."""
    rng = np.random.default_rng(1000 + s)
    U = rng.random()
    side = int(8 * round(8 * 8 ** U))
    n = int(round(32 * 8 ** U))
    spp = 4 + int(61 * U)
    if size_scale != 1.0:
        side = max(8, int(8 * round(side * size_scale / 8)))
        n = max(8, int(round(n * size_scale)))
    kind = ("sphere", "plane", "box")[int(rng.integers(0, 3))]
    bmin, bmax = (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5)
    p = node_coords(bmin, bmax, (n, n, n))
    if kind == "sphere":
        mean = sdf_sphere(p, (0, 0, 0), rng.uniform(0.2, 0.35))
    elif kind == "plane":
        mean = p[..., 2] - rng.uniform(-0.2, 0.2)
    else:
        mean = sdf_box(p, (0, 0, 0), (rng.uniform(0.15, 0.3),) * 3)
    mean = mean + 0.02 * value_noise_grid(bmin, bmax, (n, n, n), 100 + s)
    var = 1e-6 * (5e4) ** rng.random()
    obj = make_object(mean, var, 0.8, bmin, bmax, 0.01)
    return {"name": "batched_%02d" % s,
            "scene": {"objects": [obj], "light": sky_light()},
            "camera": perspective_camera(side, side),
            "opts": {"spp": spp, "max_bounces": 32, "seed": 1000 + s, "mix_R": 0.5}}


def batched(count=64, size_scale=1.0):
    return [batched_scene(s, size_scale) for s in range(count)]
