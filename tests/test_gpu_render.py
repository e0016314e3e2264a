"""GPU image parity of the forward renderer against the FP64 oracle and
against closed forms, through the C-ABI."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_00280_gb300 import gpss
from paper_2603_00280_gb300 import workloads as W
from tests import gpu_common as C
from tests import helpers as H

pytestmark = pytest.mark.gpu
D45 = np.array([math.cos(math.pi / 4), 0.0, -math.sin(math.pi / 4)])


def _gpu_render(scene_dict, cam, opts, brick=0):
    S = gpss.Scene(scene_dict, majorant_brick=brick)
    img, sq, st = gpss.render(S, cam, opts, want_sqsum=True)
    return img.cpu().numpy().astype(np.float64), sq.cpu().numpy().astype(np.float64), st


def test_single_scattering_matches_closed_form():
    """max_bounces = 1 on the plane-mean slab: every interior pixel has the exact
    value of a 1-D integral of closed forms (integrator + extinction + phase)."""
    ref = H.slab_single_scatter(D45, np.array([0.0, 0.0, 1.0]), 0.75)
    cam = W.ortho_camera_45(16, 16, film=0.5)
    spp = 16384
    for brick in (1, 4):
        img, sq, st = _gpu_render(H.dyadic_slab(albedo=0.75), cam, {"spp": spp, "max_bounces": 1, "seed": 7}, brick)
        v = img[4:12, 4:12, 0]
        se = np.sqrt(np.maximum(sq[4:12, 4:12, 0] / spp - v ** 2, 0) / spp)
        z = (v - ref) / se
        assert np.mean(np.abs(z) > 3) <= 0.05, z
        assert abs((v.mean() - ref) / (np.sqrt(np.sum(se ** 2)) / v.size)) < 4
        assert st["aborted"] == 0 and st["paths"] == 16 * 16 * spp


def test_white_furnace():
    sc = H.dyadic_slab(albedo=1.0, mean=0.0625, light=W.uniform_light(1.0))
    cam = W.ortho_camera_45(16, 16, film=0.5)
    spp = 8192
    img, sq, st = _gpu_render(sc, cam, {"spp": spp, "max_bounces": 512, "seed": 3})
    assert st["truncated"] == 0
    v = img[6:10, 6:10, 0]
    m = v.mean()
    var = sq[6:10, 6:10, 0].sum() / (16 * spp) - m * m
    se = math.sqrt(var / (16 * spp))
    assert abs(m - 1.0) < 4 * se, (m, se)


def _parity(sc, cam, opts, orc_spp, gpu_spp, rows=None, cols=None, brick=0):
    img, sq, st = _gpu_render(sc, cam, dict(opts, spp=gpu_spp, seed=101), brick)
    O = oracle.Scene(sc)
    s, s2, ost = oracle.render(O, cam, dict(opts, spp=orc_spp, seed=202, sampler="vndf"), rows=rows, cols=cols)
    H_, W_ = cam["height"], cam["width"]
    r = rows or (0, H_, 1)
    c = cols or (0, W_)
    sel = (slice(r[0], r[1], r[2] if len(r) > 2 else 1), slice(c[0], c[1]))
    z, gm, om, gse, ose = C.image_z(img[sel], sq[sel], gpu_spp, s[sel], s2[sel], orc_spp)
    ok, info = C.check_image_parity(gm, gse, om, ose)
    assert ok, info
    assert st["aborted"] == 0
    return st, ost


def test_tiny_slab_image_parity():
    """The tiny workload (64x64 orthographic view of the slab, 8 bounces) vs the oracle."""
    wl = W.tiny_slab()
    _parity(wl["scene"], wl["camera"], wl["opts"], orc_spp=128, gpu_spp=8192, rows=(0, 64, 4))


@pytest.mark.parametrize("brick", [1, 4])
def test_heterogeneous_image_parity(brick):
    wl = W.heterogeneous(n=32, width=24, height=24, spp=32, max_bounces=16)
    _parity(wl["scene"], wl["camera"], wl["opts"], orc_spp=128, gpu_spp=8192, brick=brick)


def test_rgb_albedo_and_multiple_objects_parity():
    sc = C.two_spheres_rgb()
    cam = W.perspective_camera(20, 20, eye=(0.0, -1.6, 0.6))
    _parity(sc, cam, {"spp": 16, "max_bounces": 8, "mix_R": 0.5}, orc_spp=128, gpu_spp=8192)


@pytest.mark.parametrize("sampler", ["mixture", "vndf"])
def test_zero_gradient_fog_parity(sampler):
    """A constant mean (grad mu = 0 everywhere: isotropic slopes, p = F/(4 pi)), where
    the mixture's Beckmann proposal is the roughest about -d.  A near-axis cancellation
    in the visible-normal sampler once rendered this 30% bright from the second bounce
    on; both samplers against the oracle."""
    lo, hi = (-0.125, -0.125, -0.125), (0.125, 0.125, 0.125)
    p = W.node_coords(lo, hi, (9, 9, 9))
    sc = {"objects": [W.make_object(np.full(p.shape[:3], 0.05), 0.01, 0.7, lo, hi, 0.05)], "light": W.sky_light()}
    cam = W.perspective_camera(6, 6, eye=(0.0, -1.2, 0.3), look_at=(0.0, 0.0, 0.0), fov_y_deg=12)
    st, _ = _parity(sc, cam, {"max_bounces": 4, "mix_R": 0.5, "sampler": sampler}, orc_spp=1024, gpu_spp=65536)
    assert st["vertices"] > 0


def test_tiny_brute_force_input_parity():
    """The brute-force input on which the oracle's regular tracking is checked against a
    naive delta tracker (3x3x3 nodes, 4x4 pixels, 3 bounces, directional light): the GPU
    against the oracle."""
    sc, cam, _, _ = H.tiny_brute_force_scene()
    _parity(sc, cam, {"max_bounces": 3, "mix_R": 0.5}, orc_spp=4096, gpu_spp=65536)


def test_sky_only_pixels_are_exact():
    """Rays that miss every object return the sky radiance exactly."""
    sc = C.dyadic_hetero(4)
    cam = {"type": "ortho", "eye": (3.0, 3.0, 2.0), "look_at": (4.0, 4.0, 3.0), "up": (0, 0, 1),
           "ortho_w": 0.5, "ortho_h": 0.5, "width": 8, "height": 8}
    img, sq, st = _gpu_render(sc, cam, {"spp": 4, "max_bounces": 4, "seed": 1})
    d = np.array([1.0, 1.0, 1.0]) / math.sqrt(3)
    t = d[2]
    sky = np.array([(1 - t) + t * 0.35, (1 - t) + t * 0.55, 1.0])
    np.testing.assert_allclose(img.reshape(-1, 3), np.tile(sky, (64, 1)), rtol=2e-6)
    assert st["vertices"] == 0


def test_ragged_sizes_edge_cases_and_stats():
    sc = C.dyadic_hetero(4)
    for (w, h, spp, mb) in [(37, 23, 3, 5), (1, 1, 1, 1), (33, 1, 7, 2), (5, 129, 1, 32)]:
        cam = W.perspective_camera(w, h)
        img, sq, st = _gpu_render(sc, cam, {"spp": spp, "max_bounces": mb, "seed": 9})
        assert img.shape == (h, w, 3)
        assert np.all(np.isfinite(img)) and np.all(img >= 0)
        assert st["paths"] == w * h * spp
        assert st["aborted"] == 0


def test_same_seed_same_image_and_host_output():
    wl = W.heterogeneous(n=32, width=40, height=30, spp=8, max_bounces=8)
    S = gpss.Scene(wl["scene"])
    a, _, _ = gpss.render(S, wl["camera"], wl["opts"])
    b, _, _ = gpss.render(S, wl["camera"], wl["opts"])
    host = np.zeros((30, 40, 3), np.float32)
    gpss.render(S, wl["camera"], wl["opts"], image=host)
    a = a.cpu().numpy()
    np.testing.assert_allclose(a, b.cpu().numpy(), rtol=1e-5, atol=1e-7)   # only the order of float atomics differs
    np.testing.assert_allclose(a, host, rtol=1e-5, atol=1e-7)
    c, _, _ = gpss.render(S, wl["camera"], dict(wl["opts"], seed=99))
    assert not np.allclose(a, c.cpu().numpy())


def _full_size(wl, repeats):
    """`repeats` full-size renders (the benchmark's launch) with consecutive seeds,
    combined: mean image, summed squares and the total samples per pixel."""
    S = gpss.Scene(wl["scene"])
    H_, W_, spp = wl["camera"]["height"], wl["camera"]["width"], wl["opts"]["spp"]
    m, q = np.zeros((H_, W_, 3)), np.zeros((H_, W_, 3))
    for i in range(repeats):
        img, sq, st = gpss.render(S, wl["camera"], dict(wl["opts"], seed=wl["opts"]["seed"] + 1000 * i), want_sqsum=True)
        assert st["paths"] == H_ * W_ * spp and st["aborted"] == 0
        m += img.cpu().numpy().astype(np.float64) / repeats
        q += sq.cpu().numpy().astype(np.float64)
    S.close()
    assert np.all(np.isfinite(m))
    return m, q, spp * repeats


def test_full_size_workload_sampled_pixels():
    """The heterogeneous configuration (128^3 grid, 512x512, 64 spp, 32 bounces) in
    the launch configuration the benchmark uses (16 renders with their own seeds, so
    that the GPU side's standard errors are small); a sample of pixels is checked
    against the oracle one by one."""
    wl = W.heterogeneous()
    img, sq, gspp = _full_size(wl, 16)
    O = oracle.Scene(wl["scene"])
    orc_spp = 64
    rows, cols = (220, 284, 4), (240, 256)      # 16 x 16 pixels over the sphere's shell
    s, s2, _ = oracle.render(O, wl["camera"], dict(wl["opts"], spp=orc_spp, seed=5, sampler="vndf"), rows=rows,
                             cols=cols)
    sel = (slice(*rows), slice(*cols))
    z, gm, om, gse, ose = C.image_z(img[sel], sq[sel], gspp, s[sel], s2[sel], orc_spp)
    ok, info = C.check_image_parity(gm, gse, om, ose)
    assert ok, info


def test_full_size_surface_to_volume_sampled_pixels():
    """The three-object surface-to-volume configuration at full size (torus, box and
    sphere on 256^3 grids, variances 1e-6 / 2.24e-4 / 0.05, RGB albedo; 1024x1024,
    256 spp, 64 bounces): every path completes, and sampled pixels over each object
    agree with the oracle."""
    wl = W.surface_to_volume()
    img, sq, gspp = _full_size(wl, 4)
    O = oracle.Scene(wl["scene"])
    gm_all, gse_all, om_all, ose_all = [], [], [], []
    # torus (thin shell, slow in the oracle), box, sphere: 8 x 8 pixels each
    for rows, cols, orc_spp in [((496, 504), (368, 376), 16), ((496, 504), (508, 516), 32),
                                ((496, 504), (648, 656), 32)]:
        s, s2, _ = oracle.render(O, wl["camera"], dict(wl["opts"], spp=orc_spp, seed=9, sampler="vndf"), rows=rows,
                                 cols=cols)
        sel = (slice(*rows), slice(*cols))
        z, gm, om, gse, ose = C.image_z(img[sel], sq[sel], gspp, s[sel], s2[sel], orc_spp)
        assert om.max() > 0.0  # the region sees the object
        for a, lst in ((gm, gm_all), (gse, gse_all), (om, om_all), (ose, ose_all)):
            lst.append(a.reshape(-1, 3))
    gm, gse, om, ose = (np.concatenate(l)[:, None, :] for l in (gm_all, gse_all, om_all, ose_all))
    ok, info = C.check_image_parity(gm, gse, om, ose)
    assert ok, info
