"""Pins of the oracle's transmittance and path tracer against closed forms:
constant-mean and plane-mean transmittance (Eq. sm2tr with Eq.
generalized_sigma_t), exact single scattering, a white furnace, and finite
differences with common random numbers against an exact derivative; and, on a tiny
input, against a brute-force delta/ratio tracker with one global majorant."""
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


def _box_span(o, d, lo, hi):
    """[t0, t1] of the ray o + t d inside the box [lo, hi] (t1 < t0 when it misses)."""
    t0, t1 = 0.0, math.inf
    for a in range(3):
        if d[a] == 0.0:
            if not (lo[a] <= o[a] <= hi[a]):
                return 1.0, 0.0
            continue
        ta, tb = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return t0, t1


def test_regular_tracking_agrees_with_naive_delta_tracking():
    """Brute force on a tiny input (a 3x3x3-node grid, 4x4 pixels): the oracle's path
    tracer (regular tracking: optical depth by quadrature, free-flight distance by root
    finding, transmittance by quadrature) against a textbook one written here from the
    oracle's point evaluations only -- delta tracking and ratio tracking against a single
    global majorant, the exact visible-normal sampler, next-event estimation toward a
    directional light at every vertex.  Both estimate the same image; they share no
    tracking code."""
    sc, cam, lo, hi = H.tiny_brute_force_scene()
    rng = np.random.default_rng(11)
    obj = sc["objects"][0]
    mean, var, l = obj["mean"], obj["var"], obj["length_scale"]
    O = oracle.Scene(sc)
    # global majorant: rho <= lambda(u_min)/sigma_lo with u_min the smallest mu/sigma the
    # trilinear fields reach; sigma(d) = E[max(0, -d.g)] <= |grad mu|_max + (sigma_hi/l)/sqrt(2 pi)
    m = mean.astype(np.float64)
    s_lo, s_hi = math.sqrt(float(var.min())), math.sqrt(float(var.max()))
    u_min = m.min() / (s_lo if m.min() < 0 else s_hi)
    rho_max = oracle.inv_mills(u_min) / s_lo
    h = (hi - lo) / 2.0
    gmax = math.sqrt(sum((np.abs(np.diff(m, axis=2 - a)).max() / h[a]) ** 2 for a in range(3)))
    sbar = 1.05 * rho_max * (gmax + (s_hi / l) / math.sqrt(2 * math.pi))
    wl = np.array(sc["light"]["dir"])
    bounces = 3

    def sig(x, d):
        return float(oracle.sigma_t(O, x, d)[0])

    def ratio_tracking(x, d):
        _, t1 = _box_span(x, d, lo, hi)
        T, t = 1.0, 0.0
        while True:
            t += -math.log(1.0 - rng.random()) / sbar
            if t >= t1:
                return T
            s = sig(x + t * d, d)
            assert s <= sbar
            T *= 1.0 - s / sbar

    def path(px, py):
        o, d = oracle.camera_ray(cam, px, py, rng.random(), rng.random())
        beta, L = 1.0, 0.0
        for _ in range(bounces):
            t0, t1 = _box_span(o, d, lo, hi)
            if t1 <= t0:
                return L
            t, hit = t0, False
            while True:
                t += -math.log(1.0 - rng.random()) / sbar
                if t >= t1:
                    break
                x = o + t * d
                s = sig(x, d)
                assert s <= sbar
                if rng.random() * sbar < s:
                    hit = True
                    break
            if not hit:
                return L
            pv, _ = oracle.phase_eval(O, 0, x, d, wl)
            L += beta * pv[0, 0] * ratio_tracking(x, wl)
            d2, w, _, ok = oracle.phase_sample_exact(O, 0, x, d, rng.random((1, 3)))
            if not ok[0]:
                return L
            beta *= w[0, 0]
            o, d = x, d2[0]
        return L

    n_naive = 160
    naive = np.array([[[path(px, py) for _ in range(n_naive)] for px in range(4)] for py in range(4)])
    nm, nse = naive.mean(2), naive.std(2, ddof=1) / math.sqrt(n_naive)
    spp = 4096
    s, s2, _ = oracle.render(O, cam, {"spp": spp, "max_bounces": bounces, "seed": 5, "sampler": "vndf"})
    om = s[..., 0] / spp
    ostd = np.sqrt(np.maximum(s2[..., 0] / spp - om * om, 0))
    ose = ostd / math.sqrt(spp)
    # a pixel whose few contributing paths the 160 naive samples miss shows a zero sample
    # variance: its standard error is floored at the oracle's per-path spread
    nse = np.maximum(nse, ostd / math.sqrt(n_naive))
    z = (nm - om) / np.sqrt(nse ** 2 + ose ** 2 + 1e-30)
    assert (om > 0).sum() >= 8, om
    assert np.abs(z).max() < 4, (z, nm, om)
    tot = (nm.sum() - om.sum()) / math.sqrt((nse ** 2).sum() + (ose ** 2).sum())
    assert abs(tot) < 3, (tot, nm.sum(), om.sum())


def test_zero_gradient_fog_single_scattering_closed_form():
    """A constant mean (grad mu = 0): the slopes are isotropic, so sigma(d) = alpha psi(0)
    = alpha/(2 sqrt pi) for every d, sigma_t = rho sigma(d) is constant in the box, and the
    phase function is F/(4 pi) (Eq. gdf_to_ndf with a zero mean gradient).  Single
    scattering toward a directional light is then the 1-D integral
    L = int exp(-sigma_t t) sigma_t F/(4 pi) E exp(-sigma_t s(t)) dt, s(t) the light path to
    the box face.  The oracle's extinction at such a point (every direction) and its
    rendered pixel (next-event estimation with the phase function at a zero gradient)
    against that."""
    from scipy.integrate import quad
    lo, hi = np.array([-0.125, -0.125, -0.125]), np.array([0.125, 0.125, 0.125])
    p = W.node_coords(lo, hi, (5, 5, 5))
    mu0, var0, l, F = 0.0625, 0.0078125, 0.0625, 0.75  # exact in the grids' float32
    sc = {"objects": [W.make_object(np.full(p.shape[:3], mu0), var0, F, lo, hi, l)],
          "light": W.directional_light((0.2, -0.3, 1.0), 1.0)}
    O = oracle.Scene(sc)
    sig = math.sqrt(var0)
    alpha = math.sqrt(2.0) * sig / l
    rho = oracle.inv_mills(mu0 / sig) / sig
    st = rho * alpha / (2.0 * math.sqrt(math.pi))
    rng = np.random.default_rng(3)
    for _ in range(8):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        assert oracle.sigma_t(O, [0.01, -0.02, 0.03], d)[0] == pytest.approx(st, rel=1e-12)
    wl = np.array(sc["light"]["dir"])
    cam = {"type": "ortho", "eye": (0.0, -1.0, 0.0), "look_at": (0.0, 0.0, 0.0), "up": (0.0, 0.0, 1.0),
           "fov_y_deg": 40.0, "ortho_w": 0.02, "ortho_h": 0.02, "width": 1, "height": 1}
    o = np.array([0.0, -1.0, 0.0])
    d = np.array([0.0, 1.0, 0.0])
    t0, t1 = _box_span(o, d, lo, hi)

    def f(t):
        x = o + t * d
        _, s1 = _box_span(x, wl, lo, hi)
        return math.exp(-st * (t - t0)) * st * F / (4.0 * math.pi) * math.exp(-st * s1)

    ref = quad(f, t0, t1, epsabs=0, epsrel=1e-12)[0]
    spp = 65536
    s, s2, _ = oracle.render(O, cam, {"spp": spp, "max_bounces": 1, "seed": 3})
    m = s[0, 0, 0] / spp
    se = math.sqrt(max(s2[0, 0, 0] / spp - m * m, 0.0) / spp)
    assert abs(m - ref) < 4 * se + 1e-4 * ref, (m, ref, se)
