"""The seeded synthetic inputs (paper_2603_00280_gb300/workloads.py) against the
configurations they stand in for: sizes, parameter regimes, determinism and the
structural properties both the CUDA path and the oracle rely on.  No GPU."""
import math

import numpy as np
import pytest

from paper_2603_00280_gb300 import workloads as W


def test_value_noise_is_seeded_bounded_and_grid_consistent():
    p = np.random.default_rng(0).uniform(-0.5, 0.5, size=(2000, 3))
    a, b = W.value_noise(p, 3), W.value_noise(p, 3)
    np.testing.assert_array_equal(a, b)
    assert np.abs(a).max() <= 1.0 and a.std() > 0.1
    assert np.abs(W.value_noise(p, 4) - a).max() > 0.1
    # the separable grid evaluation equals the pointwise one at the nodes
    bmin, bmax, n = (-0.5, -0.4, -0.3), (0.5, 0.6, 0.2), (9, 7, 5)
    g = W.value_noise_grid(bmin, bmax, n, 5)
    np.testing.assert_allclose(g, W.value_noise(W.node_coords(bmin, bmax, n), 5), rtol=0, atol=1e-12)


def test_node_coords_layout():
    p = W.node_coords((-1, -2, -3), (1, 2, 3), (3, 5, 7))
    assert p.shape == (7, 5, 3, 3)  # (nz, ny, nx, xyz), x fastest in memory
    np.testing.assert_allclose(p[0, 0, :, 0], [-1, 0, 1])
    np.testing.assert_allclose(p[0, :, 0, 1], np.linspace(-2, 2, 5))
    np.testing.assert_allclose(p[:, 0, 0, 2], np.linspace(-3, 3, 7))


def test_signed_distances():
    p = np.array([[0.5, 0, 0], [0, 0, 0], [1, 1, 0]], float)
    np.testing.assert_allclose(W.sdf_sphere(p, (0, 0, 0), 0.3), [0.2, -0.3, math.sqrt(2) - 0.3])
    np.testing.assert_allclose(W.sdf_box(p, (0, 0, 0), (0.2, 0.2, 0.2)), [0.3, -0.2, math.sqrt(2 * 0.8 ** 2)])
    np.testing.assert_allclose(W.sdf_torus_z(np.array([[0.25, 0, 0.0], [0.25, 0, 0.1]]), (0, 0, 0), 0.25, 0.08),
                               [-0.08, 0.02], atol=1e-15)


def test_tiny_slab_configuration():
    wl = W.tiny_slab()
    o = wl["scene"]["objects"][0]
    assert o["mean"].shape == (9, 33, 33)
    p = W.node_coords(o["bbox_min"], o["bbox_max"], (33, 33, 9))
    np.testing.assert_allclose(o["mean"], p[..., 2].astype(np.float32))  # mu = z
    assert np.all(o["var"] == np.float32(0.05 ** 2)) and o["length_scale"] == 0.02
    assert math.sqrt(2) * 0.05 / 0.02 == pytest.approx(3.536, abs=1e-3)  # alpha
    cam = wl["camera"]
    d = np.subtract(cam["look_at"], cam["eye"])
    np.testing.assert_allclose(d / np.linalg.norm(d), [math.cos(math.pi / 4), 0, -math.sin(math.pi / 4)])
    assert cam["type"] == "ortho" and (cam["width"], cam["height"]) == (64, 64)
    assert wl["scene"]["light"]["type"] == "directional" and tuple(wl["scene"]["light"]["dir"]) == (0, 0, 1)
    assert wl["opts"]["spp"] * 64 * 64 == 65536


def test_heterogeneous_configuration():
    wl = W.heterogeneous(n=32)  # the 128^3 recipe at a smaller grid
    o = wl["scene"]["objects"][0]
    p = W.node_coords(o["bbox_min"], o["bbox_max"], (32, 32, 32))
    r = np.linalg.norm(p, axis=-1)
    noise = (o["mean"] - (r - 0.3)) / 0.02
    assert np.abs(noise).max() <= 1.0 + 1e-5 and noise.std() > 0.1
    np.testing.assert_allclose(o["var"], 1e-4 + (0.01 - 1e-4) * (p[..., 0] + 0.5), rtol=1e-6)
    assert o["length_scale"] == 0.01 and np.all(o["albedo"] == np.float32(0.8))
    full = W.heterogeneous.__defaults__
    assert full[:5] == (128, 512, 512, 64, 32)
    assert wl["camera"]["eye"] == (0.0, -1.8, 0.9) and wl["scene"]["light"]["type"] == "sky"


def test_surface_to_volume_configuration():
    wl = W.surface_to_volume(n=12)
    objs = wl["scene"]["objects"]
    assert [float(o["var"].flat[0]) for o in objs] == pytest.approx([1e-6, 2.24e-4, 0.05], rel=1e-6)
    for o in objs:
        assert o["albedo"].shape[0] == 3
        assert 0.3 <= o["albedo"].min() and o["albedo"].max() <= 0.95
    full = W.surface_to_volume.__defaults__
    assert full[:5] == (256, 1024, 1024, 256, 64)


def test_differentiable_start_differs_from_the_truth_as_specified():
    gt, st = W.differentiable(n=16), W.differentiable(n=16, start=True)
    a, b = gt["scene"]["objects"][0], st["scene"]["objects"][0]
    np.testing.assert_allclose(b["var"], 2 * a["var"], rtol=1e-6)
    assert a["length_scale"] == 0.01 and b["length_scale"] == 0.012
    assert np.all(a["albedo"] == np.float32(0.8)) and np.all(b["albedo"] == np.float32(0.6))
    d = (b["mean"] - a["mean"]) / 0.01
    assert np.abs(d).max() <= 1.0 + 1e-4 and d.std() > 0.1


def test_batched_ranges():
    scenes = [W.batched_scene(s, size_scale=0.125) for s in range(64)]
    full = []
    for s in range(64):
        rng = np.random.default_rng(1000 + s)
        U = rng.random()
        full.append((int(8 * round(8 * 8 ** U)), int(round(32 * 8 ** U)), 4 + int(61 * U)))
    sides, ns, spps = zip(*full)
    assert min(sides) >= 64 and max(sides) <= 512
    assert min(ns) >= 32 and max(ns) <= 256
    assert min(spps) >= 4 and max(spps) <= 64
    var = [float(sc["scene"]["objects"][0]["var"].flat[0]) for sc in scenes]
    assert min(var) >= 1e-6 * (1 - 1e-6) and max(var) <= 0.05 * (1 + 1e-6)
    assert len(set(round(math.log10(v)) for v in var)) >= 4  # spans the range


def test_nonstationary_kernel_fields():
    wl = W.nonstationary(n=16, length_scale=0.02)
    o = wl["scene"]["objects"][0]
    p = W.node_coords(o["bbox_min"], o["bbox_max"], (16, 16, 16))
    assert o["length_scale_b"] == pytest.approx(0.04) and o["length_scale_n"] == pytest.approx(0.01)
    np.testing.assert_allclose(o["tangent"][0], -p[..., 1], atol=1e-7)
    np.testing.assert_allclose(o["tangent"][1], p[..., 0], atol=1e-7)
    assert np.all(o["tangent"][2] == np.float32(0.25))
    cs = o["correlation_scale"]
    assert cs.min() == pytest.approx(0.5) and cs.max() == pytest.approx(1.5)
    assert np.all(np.diff(cs, axis=0) > 0)  # rises from bottom (z) to top
    # unit ratios without fields leave an isotropic stationary object unchanged
    base = W.heterogeneous(n=8)["scene"]["objects"][0]
    plain = W.with_kernel(base, 1.0, 1.0, tangent=False, correlation=False)
    assert set(plain) == set(base)
