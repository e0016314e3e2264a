"""Pins of the oracle's anisotropic and non-stationary kernels (Sec. 4.2's general
gradient covariance, alpha_x, alpha_y, alpha_z in the local frame whose z axis is the
mean gradient; spatially varying correlation as in the non-stationary kernels of
Sec. 6's comparisons).  The gradient covariance is assembled here independently (the
tangent field and the correlation-scale grid interpolated with scipy), so that the
oracle's frame, its per-axis roughness and its world-to-local rotation are checked
against the definitions sigma(d) = E[max(0, -d.g)] and D(m) = int t^3 P(t m) dt."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.interpolate import RegularGridInterpolator
from scipy.stats import norm

import oracle
from paper_2603_00280_gb300 import workloads as W
from tests import helpers as H

LT = 0.05


def _object(l_b_ratio=2.0, l_n_ratio=0.5, tangent=True, correlation=True, n=9, ndf="gpss"):
    wl = W.heterogeneous(n=n, length_scale=LT)
    obj = wl["scene"]["objects"][0]
    if ndf != "gpss":
        obj = dict(obj, ndf=ndf)
    return W.with_kernel(obj, l_b_ratio, l_n_ratio, tangent, correlation), wl["scene"]["light"]


def _scene(obj, light):
    return oracle.Scene({"objects": [obj], "light": light})


def _interp(obj, grid, x):
    """Trilinear interpolation of a node grid (nz, ny, nx) at world points x (n, 3)."""
    nz, ny, nx = grid.shape
    axes = [np.linspace(obj["bbox_min"][a], obj["bbox_max"][a], (nx, ny, nz)[a]) for a in range(3)]
    f = RegularGridInterpolator((axes[2], axes[1], axes[0]), grid.astype(np.float64))
    return f(np.asarray(x)[:, ::-1])


def _covariance(obj, x, f):
    """Sigma = sigma^2 (t t^T/l_t^2 + b b^T/l_b^2 + n n^T/l_n^2) at x, every l scaled by s(x)."""
    s = _interp(obj, obj["correlation_scale"], x[None])[0] if obj.get("correlation_scale") is not None else 1.0
    lt = obj["length_scale"] * s
    lb = obj.get("length_scale_b", 0.0) or obj["length_scale"]
    ln = obj.get("length_scale_n", 0.0) or obj["length_scale"]
    lb, ln = lb * s, ln * s
    g = f["grad"]
    n = g / np.linalg.norm(g)
    if obj.get("tangent") is not None:
        t = np.array([_interp(obj, obj["tangent"][a], x[None])[0] for a in range(3)])
        t = t - (t @ n) * n
        t /= np.linalg.norm(t)
    else:
        t = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 else [0.0, 1.0, 0.0])
        t /= np.linalg.norm(t)
    b = np.cross(n, t)
    return f["var"] * (np.outer(t, t) / lt ** 2 + np.outer(b, b) / lb ** 2 + np.outer(n, n) / ln ** 2)


def _rho(f):
    sig = math.sqrt(f["var"])
    u = f["mean"] / sig
    return math.exp(norm.logpdf(u) - norm.logcdf(u)) / sig


def _points(S, seed, n, shell=0.1):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        x = rng.uniform(-0.45, 0.45, size=3)
        f = oracle.field(S, 0, x)
        if f is not None and abs(f["mean"]) < shell and np.linalg.norm(f["grad"]) > 0.1:
            out.append((x, f))
    return out


def _gauss_projected_area(d, g, Sig):
    """E[max(0, -d.g)] for g ~ N(g, Sig): the 1-D Gaussian m Phi(m/s) + s phi(m/s)."""
    m = -d @ g
    s = math.sqrt(d @ Sig @ d)
    return m * norm.cdf(m / s) + s * norm.pdf(m / s)


@pytest.fixture(scope="module")
def aniso():
    obj, light = _object()
    return obj, _scene(obj, light)


def test_projected_area_is_the_gaussian_expectation(aniso):
    """sigma_t/rho = E[max(0, -d.g)] with the covariance assembled from the tangent
    field, the three length scales and the correlation-scale factor at x."""
    obj, S = aniso
    rng = np.random.default_rng(1)
    for x, f in _points(S, 2, 25):
        Sig = _covariance(obj, x, f)
        for _ in range(4):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            want = _rho(f) * _gauss_projected_area(d, f["grad"], Sig)
            assert oracle.sigma_t(S, x, d)[0] == pytest.approx(want, rel=1e-9)


def test_ndf_is_its_definition(aniso):
    """D(m) = int_0^inf t^3 N(t m; grad mu, Sigma) dt (Eq. gdf_to_ndf), read from the
    phase function p = F D(m)/(4 sigma(d))."""
    obj, S = aniso
    rng = np.random.default_rng(3)
    for x, f in _points(S, 4, 10):
        Sig = _covariance(obj, x, f)
        Si = np.linalg.inv(Sig)
        norm_c = 1.0 / math.sqrt((2 * math.pi) ** 3 * np.linalg.det(Sig))
        g = f["grad"]
        for _ in range(3):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            # a half vector facing -d and near the mean normal (where D is not negligible)
            m = -d + 0.8 * g / np.linalg.norm(g) + 0.3 * rng.normal(size=3)
            m /= np.linalg.norm(m)
            if m @ d >= -0.05:
                continue
            d2 = d - 2 * (d @ m) * m
            p, _ = oracle.phase_eval(S, 0, x[None], d[None], d2[None])
            sd = _gauss_projected_area(d, g, Sig)
            D_oracle = 4.0 * sd * p[0, 0] / f["albedo"][0]
            A, B, C = m @ Si @ m, m @ Si @ g, g @ Si @ g
            fn = lambda t: t ** 3 * math.exp(-0.5 * (A * t * t - 2 * B * t + C))
            tm = (B + math.sqrt(B * B + 6 * A)) / (2 * A)
            w = 1 / math.sqrt(A)
            pts = sorted(set(max(0.0, tm + k * w) for k in (-8, -4, -2, 0, 2, 4, 8)))
            want = norm_c * sum(quad(fn, a, b, epsabs=0, epsrel=1e-12, limit=200)[0]
                                for a, b in zip([0.0] + pts, pts + [tm + 40 * w]) if b > a)
            assert D_oracle == pytest.approx(want, rel=1e-7, abs=1e-12 * max(want, 1.0))


def test_energy_and_reciprocity(aniso):
    """int p(d, d2) dd2 = F (the NDF integrates against max(0, -d.m) to sigma(d)) and
    sigma(d) p(d, d2) = sigma(-d2) p(-d2, -d)."""
    obj, S = aniso
    rng = np.random.default_rng(5)
    for x, f in _points(S, 6, 3):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        ms, wts = H.sphere_points(-d, 128, 128, cos_range=(0.0, 1.0))
        d2 = d - 2.0 * (ms @ d)[:, None] * ms
        xs, ds = np.repeat(x[None], len(ms), 0), np.repeat(d[None], len(ms), 0)
        p, _ = oracle.phase_eval(S, 0, xs, ds, d2)
        assert np.sum(wts * p[:, 0] * 4.0 * np.abs(ms @ d)) == pytest.approx(f["albedo"][0], rel=2e-3)
        sel = np.nonzero(p[:, 0] > 1e-3 * p[:, 0].max())[0][::97][:30]
        s1 = oracle.sigma_t(S, xs[sel], ds[sel])
        s2 = oracle.sigma_t(S, xs[sel], -d2[sel])
        p2, _ = oracle.phase_eval(S, 0, xs[sel], -d2[sel], -ds[sel])
        np.testing.assert_allclose(s1 * p[sel, 0], s2 * p2[:, 0], rtol=1e-10)


def test_near_isotropic_local_frame_route_matches_the_isotropic_form():
    """l_n = l_t (1 + 1e-9): the anisotropic route (rotation to the local frame,
    Eq. generalized_lambda and the quadrature NDF there) reproduces the isotropic
    world-frame forms."""
    iso, light = _object(1.0, 1.0, tangent=False, correlation=False)
    near = dict(iso, length_scale_n=iso["length_scale"] * (1 + 1e-9))
    Si, Sn = _scene(iso, light), _scene(near, light)
    rng = np.random.default_rng(7)
    for x, f in _points(Si, 8, 10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        d2 = rng.normal(size=3)
        d2 /= np.linalg.norm(d2)
        assert oracle.sigma_t(Sn, x, d)[0] == pytest.approx(oracle.sigma_t(Si, x, d)[0], rel=1e-8)
        pn, _ = oracle.phase_eval(Sn, 0, x[None], d[None], d2[None])
        pi, _ = oracle.phase_eval(Si, 0, x[None], d[None], d2[None])
        assert pn[0, 0] == pytest.approx(pi[0, 0], rel=1e-7, abs=1e-300)


def test_correlation_scale_is_a_local_length_scale():
    """s(x) multiplies l: a constant factor c equals the scalar l c exactly, and a
    varying factor equals, at each x, the stationary object with l s(x)."""
    base, light = _object(1.0, 1.0, tangent=False, correlation=False)
    const = dict(base, correlation_scale=np.full(base["mean"].shape, 1.25, np.float32))
    scaled = dict(base, length_scale=base["length_scale"] * 1.25)
    Sc, Ss = _scene(const, light), _scene(scaled, light)
    ramp, _ = _object(1.0, 1.0, tangent=False, correlation=True)
    Sr = _scene(ramp, light)
    rng = np.random.default_rng(9)
    for x, f in _points(Sc, 10, 8):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        d2 = rng.normal(size=3)
        d2 /= np.linalg.norm(d2)
        assert oracle.sigma_t(Sc, x, d)[0] == pytest.approx(oracle.sigma_t(Ss, x, d)[0], rel=1e-13)
        pc, _ = oracle.phase_eval(Sc, 0, x[None], d[None], d2[None])
        ps, _ = oracle.phase_eval(Ss, 0, x[None], d[None], d2[None])
        assert pc[0, 0] == pytest.approx(ps[0, 0], rel=1e-12, abs=1e-300)
        s = _interp(ramp, ramp["correlation_scale"], x[None])[0]
        Sl = _scene(dict(base, length_scale=base["length_scale"] * s), light)
        assert oracle.sigma_t(Sr, x, d)[0] == pytest.approx(oracle.sigma_t(Sl, x, d)[0], rel=1e-12)


def test_infinite_normal_correlation_is_the_beckmann_height_field():
    """Sec. 4.1: l_n -> infinity (alpha_z -> 0) with l_b = l_t turns the anisotropic
    GPSS into the Beckmann height-field macrofacet of roughness alpha_t (extinction
    and phase function), at O(alpha_z^2).  The planar mean mu = z has |grad mu| = 1
    exactly, the height field's unit slope (for |grad mu| = G the GPSS is G times the
    height field of roughness alpha_t/G)."""
    slab = H.dyadic_slab()
    plane = slab["objects"][0]
    gp = W.with_kernel(plane, 1.0, 1e4, tangent=False, correlation=True)
    hf = dict(gp, ndf="beckmann")
    del hf["length_scale_n"]  # a height field has no correlation along n
    Sg, Sh = _scene(gp, slab["light"]), _scene(hf, slab["light"])
    rng = np.random.default_rng(11)
    checked = 0
    for x, f in _points(Sg, 12, 12, shell=0.1):
        n = f["grad"] / np.linalg.norm(f["grad"])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        assert oracle.sigma_t(Sg, x, d)[0] == pytest.approx(oracle.sigma_t(Sh, x, d)[0], rel=1e-6, abs=1e-12)
        m = n + 0.3 * rng.normal(size=3)
        m /= np.linalg.norm(m)
        if m @ d >= -0.05:
            continue
        d2 = d - 2 * (d @ m) * m
        pg, _ = oracle.phase_eval(Sg, 0, x[None], d[None], d2[None])
        ph, _ = oracle.phase_eval(Sh, 0, x[None], d[None], d2[None])
        assert pg[0, 0] == pytest.approx(ph[0, 0], rel=1e-5)
        checked += 1
    assert checked >= 4


def test_ndf_first_moment_is_the_mean_gradient(aniso):
    """int m D(m) dm over the sphere = int g P(g) dg = grad mu (Eq. gdf_to_ndf with
    dg = t^2 dt dm): the world-frame NDF's first moment, independent of the projected
    area.  D(m) is read from the phase function with d = -m (so d2 = m):
    D(m) = 4 sigma(-m) p(-m, m)/F."""
    obj, S = aniso
    for x, f in _points(S, 14, 2, shell=0.05):
        g = f["grad"]
        n = g / np.linalg.norm(g)
        ms, wts = H.sphere_points(n, 384, 256)
        xs = np.repeat(x[None], len(ms), 0)
        p, _ = oracle.phase_eval(S, 0, xs, -ms, ms)
        sd = oracle.sigma_t(S, xs, -ms) / _rho(f)
        D = 4.0 * sd * p[:, 0] / f["albedo"][0]
        first = np.sum(wts[:, None] * ms * D[:, None], axis=0)
        np.testing.assert_allclose(first, g, rtol=0, atol=2e-3 * np.linalg.norm(g))
