"""Per-object traversal of scenes of several objects (gpss_scene_set_object_grids, opt-in):
rays cut at the objects' box faces walk each object's own majorant grid where one box
covers them, the union grid where boxes overlap, and skip the space between boxes.
Ratio tracking and free-flight sampling stay unbiased across every kind of interval
(against the FP64 oracle's transmittance), images agree with the oracle and with the
union-grid traversal, and the thin object's local majorants cut its null collisions."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_00280_gb300 import gpss
from paper_2603_00280_gb300 import workloads as W
from tests import gpu_common as C

pytestmark = pytest.mark.gpu


def three_objects():
    """A thick sphere on a coarse grid (h = 1/32, sigma 0.063), a surface-like sphere on
    a fine grid (h = 1/64, sigma = 2^-9: local majorants on its own grid), and a fog block
    whose box overlaps the first sphere's box over x in [-0.25, -0.125]."""
    objs = []
    lo, hi = (-0.625, -0.25, -0.25), (-0.125, 0.25, 0.25)
    p = W.node_coords(lo, hi, (17, 17, 17))
    objs.append(W.make_object(W.sdf_sphere(p, (-0.375, 0.0, 0.0), 0.2), 4e-3, 0.8, lo, hi, 0.05))
    lo, hi = (0.125, -0.25, -0.25), (0.625, 0.25, 0.25)
    p = W.node_coords(lo, hi, (33, 33, 33))
    objs.append(W.make_object(W.sdf_sphere(p, (0.375, 0.0, 0.0), 0.2), 2.0 ** -18, 0.9, lo, hi, 0.01))
    lo, hi = (-0.25, -0.125, -0.125), (0.0, 0.125, 0.125)
    p = W.node_coords(lo, hi, (9, 9, 9))
    objs.append(W.make_object(np.full(p.shape[:3], 0.05), 0.01, 0.7, lo, hi, 0.05))
    return {"objects": objs, "light": W.sky_light()}


@pytest.fixture(scope="module")
def scene():
    sc = three_objects()
    return sc, gpss.Scene(sc), oracle.Scene(sc)


def _rays():
    """Group 1: along +x past the spheres' shells (one-box intervals and the gap between
    the boxes), full length.  Group 2: from the overlap of the thick sphere's box and the
    fog block (a union-grid interval), through the fog alone and the gap, ending inside
    the thin sphere's box before its shell."""
    rng = np.random.default_rng(17)
    n1, n2 = 32, 16
    o1 = np.stack([np.full(n1, -0.9), rng.uniform(0.17, 0.27, n1), rng.uniform(-0.05, 0.05, n1)], 1)
    d1 = np.stack([np.ones(n1), rng.uniform(-0.02, 0.02, n1), rng.uniform(-0.02, 0.02, n1)], 1)
    o2 = np.stack([np.full(n2, -0.15), rng.uniform(-0.08, 0.08, n2), rng.uniform(-0.08, 0.08, n2)], 1)
    d2 = np.stack([np.ones(n2), rng.uniform(-0.1, 0.1, n2), rng.uniform(-0.1, 0.1, n2)], 1)
    o = np.concatenate([o1, o2]).astype(np.float32)
    d = np.concatenate([d1, d2])
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    tmax = np.concatenate([np.full(n1, np.inf), np.full(n2, 0.3)]).astype(np.float32)
    return o, d, tmax


@pytest.mark.parametrize("object_grids", [True, False])
def test_ratio_tracking_unbiased_across_boxes(scene, object_grids):
    sc, G, O = scene
    G.set_object_grids(object_grids)
    o, d, tmax = _rays()
    n = len(o)
    ref = np.array([oracle.transmittance(O, o[i].astype(np.float64), d[i].astype(np.float64), float(tmax[i]))
                    for i in range(n)])
    assert ((ref > 0.05) & (ref < 0.95)).sum() > 12, ref
    N = 40000
    m = gpss.estimate_transmittance(G, o, d, tmax, N, seed=3).cpu().numpy().astype(np.float64)
    se = np.sqrt(np.maximum(ref * (1 - ref), 1e-4) / N)
    z = (m - ref) / se
    G.set_object_grids(False)
    assert np.mean(np.abs(z) > 4) < 0.05, z
    assert abs(np.sum(m - ref)) < 4 * np.sqrt(np.sum(se ** 2)), (np.sum(m - ref), z)


@pytest.mark.parametrize("object_grids", [True, False])
def test_free_flight_distribution_across_boxes(scene, object_grids):
    """P(t_hit <= s) = 1 - Tr(s) for a ray that starts where two boxes overlap and runs
    through the fog alone, the gap and into the thin sphere."""
    sc, G, O = scene
    G.set_object_grids(object_grids)
    o = np.array([[-0.15, 0.03, 0.01]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)
    n = 200000
    t = gpss.sample_free_flight(G, o, d, n, seed=9).cpu().numpy()[0]
    G.set_object_grids(False)
    for s in (0.01, 0.05, 0.1, 0.15, 0.3, 0.33, 0.34, 0.36):
        p = float(np.mean(t <= s))
        ref = 1 - oracle.transmittance(O, o[0].astype(np.float64), d[0].astype(np.float64), s)
        assert abs(p - ref) < 5 * math.sqrt(max(ref * (1 - ref), 1e-8) / n) + 1e-4, (object_grids, s, p, ref)


def _img(G, cam, opts):
    img, sq, st = gpss.render(G, cam, opts, want_sqsum=True)
    return img.cpu().numpy().astype(np.float64), sq.cpu().numpy().astype(np.float64), st


def test_images_object_grids_vs_union_grid(scene):
    """Both traversals render the same image (independent seeds, 3 SE bar); the thin
    sphere's local majorants on its own grid cut the null collisions."""
    sc, G, _ = scene
    cam = W.perspective_camera(24, 24, eye=(0.0, -1.7, 0.5))
    spp = 2048
    opts = {"spp": spp, "max_bounces": 8, "sampler": "vndf"}
    G.set_object_grids(True)
    a, asq, sa = _img(G, cam, dict(opts, seed=41))
    G.set_object_grids(False)
    b, bsq, sb = _img(G, cam, dict(opts, seed=42))
    z, gm, om, gse, ose = C.image_z(a, asq, spp, b * spp, bsq, spp)
    ok, info = C.check_image_parity(gm, gse, om, ose)
    assert ok, info
    assert sa["aborted"] == 0 and sb["aborted"] == 0
    assert sa["null_collisions"] < 0.5 * sb["null_collisions"], (sa["null_collisions"], sb["null_collisions"])


def test_image_parity_oracle(scene):
    sc, G, O = scene
    cam = W.perspective_camera(8, 8, eye=(0.0, -1.7, 0.5))
    opts = {"max_bounces": 4, "mix_R": 0.5}
    G.set_object_grids(True)
    img, sq, st = _img(G, cam, dict(opts, spp=32768, seed=51))
    G.set_object_grids(False)
    s, s2, ost = oracle.render(O, cam, dict(opts, spp=128, seed=52, sampler="vndf"))
    z, gm, om, gse, ose = C.image_z(img, sq, 32768, s, s2, 128)
    ok, info = C.check_image_parity(gm, gse, om, ose)
    assert ok, info
    assert st["aborted"] == 0
