"""Pins of the oracle's transmittance and path tracer against closed forms:
constant-mean and plane-mean transmittance (Eq. sm2tr with Eq.
generalized_sigma_t), exact single scattering, a white furnace, and finite
differences with common random numbers against an exact derivative."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_00280_gb300 import workloads as W
from tests import helpers as H

D45 = np.array([math.cos(math.pi / 4), 0.0, -math.sin(math.pi / 4)])


def test_constant_mean_transmittance_is_exponential():
    """grad mu = 0: sigma(d) = alpha/(2 sqrt(pi)) in every direction and
    sigma_t = lambda(mu/sigma)/sigma * sigma(d) is constant: Tr = exp(-sigma_t L)."""
    S = oracle.Scene(H.dyadic_slab(mean=0.0625))
    sig = H.SLAB_SIGMA
    alpha = math.sqrt(2) * sig / H.SLAB_L
    st = oracle.inv_mills(0.0625 / sig) / sig * alpha / (2 * math.sqrt(math.pi))
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        o = np.array([0.1, -0.2, 0.0])
        t_exit = min((0.125 - o[2] * np.sign(d[2])) / abs(d[2]), (0.5 - abs(o[0])) / max(abs(d[0]), 1e-9),
                     (0.3) / max(abs(d[1]), 1e-9))
        L = 0.99 * t_exit * rng.random()
        assert oracle.transmittance(S, o, d, L) == pytest.approx(math.exp(-st * L), rel=1e-12)
        assert oracle.sigma_t(S, o, d)[0] == pytest.approx(st, rel=1e-13)


@pytest.mark.parametrize("dz", [-0.95, -math.sqrt(0.5), -0.3, 0.4, math.sqrt(0.5), 0.9])
def test_plane_mean_transmittance_closed_form(dz):
    """mu = z: int lambda(u) du = ln Phi(u) gives
    Tr = (Phi(u0)/Phi(u1))^(sigma(d)/d_z) (Smith's G1 for the height field,
    Sec. 4.1); checked along the ray at several distances, including the
    paper's 45 degree geometry."""
    S = oracle.Scene(H.dyadic_slab())
    d = np.array([math.sqrt(1 - dz * dz), 0.0, dz])
    o = np.array([-0.45, 0.0, 0.125 if dz < 0 else -0.125])
    tmax = 0.25 / abs(dz)
    for f in (0.1, 0.35, 0.6, 0.999):
        t = f * tmax
        z1 = o[2] + t * dz
        ref = H.slab_optical_depth(o[2], z1, d)
        assert oracle.optical_depth(S, o, d, t) == pytest.approx(ref, rel=1e-11)


def test_single_scattering_is_exact():
    """max_bounces = 1 with a directional light: every interior pixel of the
    orthographic 45 degree view has the same exact value, a 1-D integral of
    closed forms (transmittance both ways, constant phase function)."""
    wl = np.array([0.0, 0.0, 1.0])
    S = oracle.Scene(H.dyadic_slab(albedo=0.75))
    cam = W.ortho_camera_45(16, 16, film=0.5)
    ref = H.slab_single_scatter(D45, wl, 0.75)
    spp = 1024
    s, s2, st = oracle.render(S, cam, {"spp": spp, "max_bounces": 1, "seed": 3}, rows=(4, 12, 1), cols=(4, 12))
    v = s[4:12, 4:12, 0] / spp
    se = np.sqrt(np.maximum(s2[4:12, 4:12, 0] / spp - v ** 2, 0) / spp)
    z = H.zscores(v, se, ref)
    assert np.mean(np.abs(z) > 3) <= 0.03
    zall = (v.mean() - ref) / math.sqrt(np.sum(se ** 2)) * v.size / v.size
    assert abs((v.mean() - ref) / (np.sqrt(np.sum(se ** 2)) / v.size)) < 3.5
    assert st["truncated"] == st["vertices"]


@pytest.mark.parametrize("sampler", ["mixture", "vndf"])
def test_white_furnace(sampler):
    """Albedo 1 under a uniform unit environment: every pixel equals 1 when no
    path is truncated (energy conservation of Eq. phase and the integrator), with
    the paper's sampling mixture and with exact visible-normal sampling."""
    S = oracle.Scene(H.dyadic_slab(albedo=1.0, mean=0.0625, light=W.uniform_light(1.0)))
    cam = W.ortho_camera_45(16, 16, film=0.5)
    spp = 2048
    s, s2, st = oracle.render(S, cam, {"spp": spp, "max_bounces": 512, "seed": 9, "sampler": sampler},
                              rows=(6, 10, 1), cols=(6, 10))
    assert st["truncated"] == 0
    n = 16 * spp
    m = s[6:10, 6:10, 0].sum() / n
    se = math.sqrt((s2[6:10, 6:10, 0].sum() / n - m * m) / n)
    assert abs(m - 1.0) < 4 * se, (m, se)
    assert np.allclose(s[6:10, 6:10, 0], s[6:10, 6:10, 1])


@pytest.mark.parametrize("which", ["length_scale", "variance"])
def test_crn_finite_difference_matches_exact_derivative(which):
    """The oracle's gradient reference (central differences of renders with
    common random numbers) against the derivative of the exact single-scatter
    value."""
    wl = np.array([0.0, 0.0, 1.0])
    sig, l = H.SLAB_SIGMA, H.SLAB_L
    rel = 1e-2
    if which == "length_scale":
        kp, km = dict(l=l * (1 + rel)), dict(l=l * (1 - rel))
        h = 2 * l * rel
    else:
        kp, km = dict(sigma=sig * math.sqrt(1 + rel)), dict(sigma=sig * math.sqrt(1 - rel))
        h = 2 * sig * sig * rel
    exact = (H.slab_single_scatter(D45, wl, 0.75, **kp) - H.slab_single_scatter(D45, wl, 0.75, **km)) / h
    Sp = oracle.Scene(H.dyadic_slab(albedo=0.75, **kp))
    Sm = oracle.Scene(H.dyadic_slab(albedo=0.75, **km))
    cam = W.ortho_camera_45(16, 16, film=0.5)
    spp = 512
    s, s2, _ = oracle.render_diff(Sp, Sm, cam, {"spp": spp, "max_bounces": 1, "seed": 4}, rows=(6, 10, 1), cols=(6, 10))
    n = 16 * spp
    m = s[6:10, 6:10, 0].sum() / n / h
    se = math.sqrt(max(s2[6:10, 6:10, 0].sum() / n - (m * h) ** 2, 0) / n) / h
    assert abs(m - exact) < 4 * se + 1e-3 * abs(exact), (m, se, exact)
    assert se < 0.05 * abs(exact)


def test_orthographic_camera_convention():
    cam = W.ortho_camera_45(4, 2, film=1.0)
    o, d = oracle.camera_ray(cam, 0, 0, 0.5, 0.5)
    np.testing.assert_allclose(d, D45, atol=1e-15)
    # right = d x up = (0,-1,0); image up = right x d
    right = np.array([0.0, -1.0, 0.0])
    up = np.cross(right, D45)
    x, y = 2 * 0.5 / 4 - 1, 1 - 2 * 0.5 / 2
    np.testing.assert_allclose(o, -2 * D45 + x * 0.5 * right + y * 0.5 * up, atol=1e-15)


def test_two_objects_choose_the_scatterer_by_extinction():
    """Several objects (reading Q13): extinctions add, and a real collision scatters
    off object k with probability sigma_t,k/sigma_t.  Two co-located plane-mean
    objects with different variances, length scales and albedos: the single-
    scattered radiance is exactly int T (sigma_t,A p_A + sigma_t,B p_B) T_L dt, a 1-D
    integral of closed forms.  A uniform choice of the object would converge to
    0.90x of it here, always the first object to 1.23x, always the second to 0.57x."""
    objs = [(0.9, H.SLAB_SIGMA, H.SLAB_L), (0.2, 0.125, 0.25)]
    a = H.dyadic_slab(albedo=objs[0][0], sigma=objs[0][1], l=objs[0][2])["objects"][0]
    b = H.dyadic_slab(albedo=objs[1][0], sigma=objs[1][1], l=objs[1][2])["objects"][0]
    S = oracle.Scene({"objects": [a, b], "light": W.directional_light((0.0, 0.0, 1.0), 1.0)})
    ref = H.slab_single_scatter_objects(D45, np.array([0.0, 0.0, 1.0]), objs)
    cam = W.ortho_camera_45(16, 16, film=0.5)
    spp = 2048
    s, s2, st = oracle.render(S, cam, {"spp": spp, "max_bounces": 1, "seed": 21}, rows=(6, 10, 1), cols=(6, 10))
    v = s[6:10, 6:10, 0] / spp
    se = np.sqrt(np.maximum(s2[6:10, 6:10, 0] / spp - v ** 2, 0) / spp)
    se_mean = np.sqrt(np.sum(se ** 2)) / v.size
    assert abs(v.mean() - ref) < 4 * se_mean, (v.mean(), ref, se_mean)
    assert se_mean < 0.015 * ref  # a uniform choice (10% off) fails by more than 6 SE


@pytest.mark.parametrize("tau", [100.0, 600.0, 740.0, 800.0, 5000.0, 20000.0])
def test_transmittance_across_the_underflow_cutoff(tau):
    """The oracle stops integrating once a rough optical depth exceeds 1e4, where
    exp(-tau) is exactly 0 in double precision: on a constant-mean slab (sigma_t
    constant, Tr = exp(-sigma_t L)) the returned transmittance equals the closed
    form on both sides of underflow (tau = 745) and of the cut-off."""
    sig, l, mu = 2.0 ** -8, 2.0 ** -11, -0.125
    S = oracle.Scene(H.dyadic_slab(mean=mu, sigma=sig, l=l))
    alpha = math.sqrt(2) * sig / l
    st = oracle.inv_mills(mu / sig) / sig * alpha / (2 * math.sqrt(math.pi))
    assert st > 1e4  # a unit length is beyond the cut-off
    o = np.array([-0.45, 0.0, 0.0])
    d = np.array([1.0, 0.0, 0.0])
    L = tau / st
    assert L < 0.9
    ref = math.exp(-st * L)
    got = oracle.transmittance(S, o, d, L)
    if ref > 1e-300:
        assert got == pytest.approx(ref, rel=1e-9)
    else:
        assert abs(got - ref) <= 1e-320
    assert oracle.optical_depth(S, o, d, L) == pytest.approx(st * L, rel=1e-11)


def test_exact_sampler_and_mixture_render_the_same_image():
    """Multi-bounce heterogeneous scene: the oracle's two phase samplers are
    estimators of the same image (pixel sums over the image agree within their
    standard errors), and the exact sampler's per-path variance is far lower."""
    wl = W.heterogeneous(n=16, width=8, height=8, spp=64, max_bounces=8, length_scale=0.03)
    S = oracle.Scene(wl["scene"])
    out = {}
    for sampler, spp in (("mixture", 256), ("vndf", 256)):
        s, s2, _ = oracle.render(S, wl["camera"], dict(wl["opts"], spp=spp, seed=31, sampler=sampler))
        m = s[..., 0] / spp
        var = np.maximum(s2[..., 0] / spp - m * m, 0)
        out[sampler] = (m.sum(), math.sqrt(var.sum() / spp), var.sum())
    (a, sa, va), (b, sb, vb) = out["mixture"], out["vndf"]
    assert abs(a - b) < 4 * math.sqrt(sa * sa + sb * sb), (a, sa, b, sb)
    assert vb < 0.5 * va
