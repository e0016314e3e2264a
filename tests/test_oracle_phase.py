"""Pins of the oracle's phase function and its sampling mixture (Eq. phase,
Eq. microfacet_vndf and the mixture at the end of Sec. 4.2)."""
import math

import numpy as np
import pytest
from scipy.stats import chisquare

import oracle
from paper_2603_00280_gb300 import workloads as W
from tests import helpers as H


@pytest.fixture(scope="module")
def hetero():
    wl = W.heterogeneous(n=16)
    return oracle.Scene(wl["scene"])


@pytest.fixture(scope="module")
def moderate():
    """Roughness 0.3..3 (l = 0.05), where a product rule resolves the Beckmann vNDF."""
    wl = W.heterogeneous(n=16, length_scale=0.05)
    return oracle.Scene(wl["scene"])


def _points(seed, n):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.4, 0.4, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d2 = rng.normal(size=(n, 3))
    d2 /= np.linalg.norm(d2, axis=1, keepdims=True)
    return x, d, d2


def test_reciprocity(hetero):
    """sigma_t(x,d) p(d,d2) = sigma_t(x,-d2) p(-d2,-d): the medium's scattering
    kernel is symmetric (the paper states reciprocity for Eq. phase)."""
    x, d, d2 = _points(1, 40)
    p1, _ = oracle.phase_eval(hetero, 0, x, d, d2)
    p2, _ = oracle.phase_eval(hetero, 0, x, -d2, -d)
    s1 = oracle.sigma_t(hetero, x, d)
    s2 = oracle.sigma_t(hetero, x, -d2)
    np.testing.assert_allclose(s1[:, None] * p1, s2[:, None] * p2, rtol=1e-11, atol=1e-300)


def _reflect(d, m):
    return d - 2.0 * (d @ m) * m


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_energy_and_pdf_normalisation(moderate, seed):
    """int p(d,d2) dd2 = F and int pdf(d2) dd2 = 1, integrated over half-vectors
    m on the hemisphere facing -d with the Jacobian dd2 = 4|d.m| dm."""
    hetero = moderate
    x, d, _ = _points(seed, 1)
    x, d = x[0], d[0]
    F = oracle.field(hetero, 0, x)["albedo"][0]
    ms, wts = H.sphere_points(-d, 96, 96, cos_range=(0.0, 1.0))
    d2 = np.array([_reflect(d, m) for m in ms])
    p, pdf = oracle.phase_eval(hetero, 0, np.repeat(x[None], len(ms), 0), np.repeat(d[None], len(ms), 0), d2)
    jac = 4.0 * np.abs(ms @ d)
    assert np.sum(wts * p[:, 0] * jac) == pytest.approx(F, rel=2e-4)
    assert np.sum(wts * pdf * jac) == pytest.approx(1.0, rel=2e-4)


def test_sampler_histogram_matches_pdf(hetero):
    """chi^2 of sampled half-vectors against the mixture pdf integrated over bins,
    and the returned weight equals p/pdf at the sampled direction."""
    x, d, _ = _points(5, 1)
    x, d = x[0], d[0]
    n = 20000
    rng = np.random.default_rng(6)
    u = rng.random((n, 3))
    d2, w, pdf, ok = oracle.phase_sample(hetero, 0, np.repeat(x[None], n, 0), np.repeat(d[None], n, 0), u)
    assert ok.all()
    m = d2 - d
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    fx, fy, fz = H.frame(-d)
    c = m @ fz
    ph = np.mod(np.arctan2(m @ fy, m @ fx), 2 * math.pi)
    nc, nphi = 8, 8
    obs, _, _ = np.histogram2d(c, ph, bins=[np.linspace(0, 1, nc + 1), np.linspace(0, 2 * math.pi, nphi + 1)])
    # expected bin probabilities by 8x8 Gauss-Legendre inside each bin
    gx, gw = np.polynomial.legendre.leggauss(8)
    exp_p = np.zeros((nc, nphi))
    for i in range(nc):
        cc = (i + 0.5 + 0.5 * gx) / nc
        cw = 0.5 * gw / nc
        for j in range(nphi):
            pp = (j + 0.5 + 0.5 * gx) * 2 * math.pi / nphi
            pw = 0.5 * gw * 2 * math.pi / nphi
            CC, PP = np.meshgrid(cc, pp, indexing="ij")
            WW = np.outer(cw, pw)
            s = np.sqrt(1 - CC ** 2)
            mm = (s * np.cos(PP))[..., None] * fx + (s * np.sin(PP))[..., None] * fy + CC[..., None] * fz
            mm = mm.reshape(-1, 3)
            dd2 = np.array([_reflect(d, q) for q in mm])
            _, pdf_b = oracle.phase_eval(hetero, 0, np.repeat(x[None], len(mm), 0), np.repeat(d[None], len(mm), 0), dd2)
            exp_p[i, j] = np.sum(WW.reshape(-1) * pdf_b * 4 * np.abs(mm @ d))
    assert exp_p.sum() == pytest.approx(1.0, rel=1e-3)
    stat, pval = chisquare(obs.ravel(), exp_p.ravel() / exp_p.sum() * n)
    assert pval > 1e-4, (stat, pval)
    # weight consistency and unbiasedness of E[weight] = F
    pe, pdfe = oracle.phase_eval(hetero, 0, np.repeat(x[None], 50, 0), np.repeat(d[None], 50, 0), d2[:50])
    np.testing.assert_allclose(pdf[:50], pdfe, rtol=1e-9)
    np.testing.assert_allclose(w[:50, 0], pe[:, 0] / pdfe, rtol=1e-9)
    F = oracle.field(hetero, 0, x)["albedo"][0]
    assert abs(w[:, 0].mean() - F) < 4 * w[:, 0].std() / math.sqrt(n)


def _hist_chi2(scene, x, d, d2, pdf_fn, nc=8, nphi=8):
    """chi^2 p-value of sampled half vectors (from d2) against a pdf over d2, with the
    expected bin probabilities by 8x8 Gauss-Legendre per (cos, phi) bin about -d."""
    n = len(d2)
    m = d2 - d
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    fx, fy, fz = H.frame(-d)
    c = m @ fz
    ph = np.mod(np.arctan2(m @ fy, m @ fx), 2 * math.pi)
    obs, _, _ = np.histogram2d(c, ph, bins=[np.linspace(0, 1, nc + 1), np.linspace(0, 2 * math.pi, nphi + 1)])
    gx, gw = np.polynomial.legendre.leggauss(8)
    exp_p = np.zeros((nc, nphi))
    for i in range(nc):
        cc = (i + 0.5 + 0.5 * gx) / nc
        cw = 0.5 * gw / nc
        for j in range(nphi):
            pp = (j + 0.5 + 0.5 * gx) * 2 * math.pi / nphi
            pw = 0.5 * gw * 2 * math.pi / nphi
            CC, PP = np.meshgrid(cc, pp, indexing="ij")
            WW = np.outer(cw, pw)
            s = np.sqrt(1 - CC ** 2)
            mm = ((s * np.cos(PP))[..., None] * fx + (s * np.sin(PP))[..., None] * fy + CC[..., None] * fz).reshape(-1, 3)
            dd2 = np.array([_reflect(d, q) for q in mm])
            exp_p[i, j] = np.sum(WW.reshape(-1) * pdf_fn(dd2) * 4 * np.abs(mm @ d))
    assert exp_p.sum() == pytest.approx(1.0, rel=2e-3)
    e = exp_p.ravel() / exp_p.sum() * n
    o = obs.ravel()
    small = e < 5  # bins the density (nearly) never reaches are pooled into one
    if small.any():
        e = np.append(e[~small], e[small].sum())
        o = np.append(o[~small], o[small].sum())
        if e[-1] < 1e-9:
            assert o[-1] == 0
            e, o = e[:-1], o[:-1]
    return chisquare(o, e * o.sum() / e.sum())[1]


def _exact_cases():
    wl = W.heterogeneous(n=16, length_scale=0.05)
    iso = wl["scene"]
    obj = dict(iso["objects"][0])
    aniso = {"objects": [W.with_kernel(obj, tangent=True, correlation=True)], "light": iso["light"]}
    p = W.node_coords((-0.5, -0.5, -0.25), (0.5, 0.5, 0.25), (9, 9, 9))
    hf = {"objects": [dict(W.make_object(p[..., 2] + 0.05 * np.sin(4 * p[..., 0]), 0.02 ** 2, 0.7, (-0.5, -0.5, -0.25),
                                         (0.5, 0.5, 0.25), 0.05), ndf="beckmann")], "light": iso["light"]}
    return {"gpss": iso, "anisotropic": aniso, "beckmann": hf}


@pytest.mark.parametrize("case", ["gpss", "anisotropic", "beckmann"])
@pytest.mark.parametrize("side", ["approaching", "leaving"])
def test_exact_visible_normal_sampler(case, side):
    """The oracle's exact visible-normal sampler (slope-space sampling, visible slope
    by bisection of its closed-form CDF): the returned weight is F and the pdf is p/F
    at the sampled direction, and a chi^2 test of the sampled half vectors against
    p/F (the oracle's phase function, quadrature of the NDF's definition) holds, for
    rays approaching (beta > 0) and leaving (beta < 0) the mean surface."""
    sc = _exact_cases()[case]
    S = oracle.Scene(sc)
    rng = np.random.default_rng(11)
    while True:
        x = rng.uniform(-0.3, 0.3, 3) if case != "beckmann" else np.array([0.1, -0.05, 0.01])
        f = oracle.field(S, 0, x)
        if abs(f["mean"]) < 0.1:
            break
    nrm = f["grad"] / np.linalg.norm(f["grad"])
    d = -0.6 * nrm + 0.8 * H.frame(nrm)[0] if side == "approaching" else 0.5 * nrm + 0.866 * H.frame(nrm)[1]
    d /= np.linalg.norm(d)
    if case == "beckmann" and side == "leaving":
        d = -0.3 * nrm + 0.954 * H.frame(nrm)[1]  # height fields sample uniformly from below; stay above
        d /= np.linalg.norm(d)
    n = 20000
    u = np.random.default_rng(12).random((n, 3))
    d2, w, pdf, ok = oracle.phase_sample_exact(S, 0, np.repeat(x[None], n, 0), np.repeat(d[None], n, 0), u)
    assert ok.mean() > 0.999
    d2, w, pdf = d2[ok], w[ok], pdf[ok]
    np.testing.assert_allclose(w, np.repeat(f["albedo"][None], len(w), 0), rtol=1e-12)
    pe, _ = oracle.phase_eval(S, 0, np.repeat(x[None], 64, 0), np.repeat(d[None], 64, 0), d2[:64])
    np.testing.assert_allclose(pdf[:64], pe[:, 0] / f["albedo"][0], rtol=1e-10)

    def pdf_fn(dd2):
        pv, _ = oracle.phase_eval(S, 0, np.repeat(x[None], len(dd2), 0), np.repeat(d[None], len(dd2), 0), dd2)
        return pv[:, 0] / f["albedo"][0]

    assert _hist_chi2(S, x, d, d2, pdf_fn) > 1e-4


@pytest.mark.parametrize("sampler", ["mixture", "exact"])
def test_samplers_at_a_zero_mean_gradient(sampler):
    """A constant mean (grad mu = 0): the phase function is isotropic, F/(4 pi), so
    weighted samples must be spread uniformly in cos(d, d2) and in azimuth about d, with
    mean weight F.  (The mixture's Beckmann proposal is then the roughest, about -d.)"""
    lo, hi = (-0.125, -0.125, -0.125), (0.125, 0.125, 0.125)
    p = W.node_coords(lo, hi, (5, 5, 5))
    F = 0.75
    O = oracle.Scene({"objects": [W.make_object(np.full(p.shape[:3], 0.0625), 0.0078125, F, lo, hi, 0.0625)]})
    x = np.array([0.01, -0.02, 0.03])
    d = np.array([0.3, 0.5, -0.8])
    d /= np.linalg.norm(d)
    n = 40000
    u = np.random.default_rng(5).random((n, 3))
    xs, ds = np.tile(x, (n, 1)), np.tile(d, (n, 1))
    if sampler == "exact":
        d2, w, pdf, ok = oracle.phase_sample_exact(O, 0, xs, ds, u)
    else:
        d2, w, pdf, ok = oracle.phase_sample(O, 0, xs, ds, u)
    assert ok.mean() > 0.999
    w = w[:, 0] * ok
    assert abs(w.mean() - F) < 5 * w.std() / math.sqrt(n) + 1e-12, (w.mean(), F)
    c = d2 @ d
    fx, fy, _ = H.frame(d)
    ph = np.mod(np.arctan2(d2 @ fy, d2 @ fx), 2 * math.pi)
    # weighted counts in (cos, azimuth) cells against F/(4 pi) x the cell's solid angle
    nb = 6
    ci = np.clip(((c + 1) / 2 * nb).astype(int), 0, nb - 1)
    pj = np.clip((ph / (2 * math.pi) * nb).astype(int), 0, nb - 1)
    cells = np.zeros((nb, nb))
    np.add.at(cells, (ci, pj), w)
    expect = F * n / (nb * nb)
    se = np.sqrt(np.zeros_like(cells) + (w ** 2).mean() * n / (nb * nb))  # Poisson-like cell counts
    z = (cells - expect) / se
    assert np.abs(z).max() < 4.5, z
    # the pdf is the density of the returned directions: the exact sampler's is p/F = 1/(4 pi)
    if sampler == "exact":
        assert np.allclose(pdf[ok], 1.0 / (4 * math.pi), rtol=1e-9)
