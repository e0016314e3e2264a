"""Surface-limit analytic free flight (linear-exponential local majorants): the
piece's closed-form optical depth, its inversion and its majorant agree with each
other (d tau/dt = the majorant at the sampled point), the majorant bounds sigma_t, and
free flight, ratio tracking and images stay unbiased against the FP64 oracle and
against constant local pieces, with fewer tentative collisions."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_00280_gb300 import gpss
from paper_2603_00280_gb300 import workloads as W
from tests import gpu_common as C
from tests.test_gpu_thin_shell import thin_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plane():
    sc = thin_scene("plane")
    return sc, gpss.Scene(sc), oracle.Scene(sc)


@pytest.fixture(scope="module")
def sphere():
    sc = thin_scene("sphere", n=33, var=2.0 ** -18)
    return sc, gpss.Scene(sc), oracle.Scene(sc)


def _receding_rays(O, which, n, seed, sigma):
    """Rays leaving the shell at grazing angles (where a linear-exponential piece has a
    non-negligible depth): a shell point (the crossing of mu = 0 along a vertical line
    through the plane, or a radial line of the sphere, by bisection on the oracle's
    mean), moved along the normal to mu = c sigma with c in [-3, 1], with a direction
    whose rise rate d.grad mu lies in [0.02, 0.3]."""
    rng = np.random.default_rng(seed)
    os_, ds_ = [], []
    while len(os_) < n:
        if which == "plane":
            a = np.array([rng.uniform(-0.35, 0.35), rng.uniform(-0.35, 0.35), 0.2])
            b = a - np.array([0.0, 0.0, 0.4])
        else:
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            a, b = 0.45 * u, 0.1 * u
        lo, hi = 0.0, 1.0
        for _ in range(40):
            mid = 0.5 * (lo + hi)
            f = oracle.field(O, 0, a + mid * (b - a))
            if f is None or f["mean"] > 0.0:
                lo = mid
            else:
                hi = mid
        x = a + lo * (b - a)
        g = oracle.field(O, 0, x)["grad"]
        G = np.linalg.norm(g)
        nrm = g / G
        x = x + rng.uniform(-3.0, 1.0) * sigma / G * nrm
        t = np.cross(nrm, rng.normal(size=3))
        t /= np.linalg.norm(t)
        c = rng.uniform(0.02, 0.3) / G
        os_.append(x)
        ds_.append(c * nrm + math.sqrt(1 - c * c) * t)
    return np.array(os_, np.float32), np.array(ds_, np.float32)


@pytest.mark.parametrize("which", ["plane", "sphere"])
def test_piece_depth_inversion_and_bound(which, request):
    """Linear-exponential pieces of rays leaving the shell: monotone collisions in tau,
    d tau/dt = the majorant (trapezoid over 257 depths), the majorant above sigma_t at
    every sampled point, and few expected null collisions per piece."""
    sc, G, O = request.getfixturevalue(which)
    sigma = math.sqrt(float(sc["objects"][0]["var"].flat[0]))
    n, k = 384, 257
    o, d = _receding_rays(O, which, n, 3 if which == "plane" else 4, sigma)
    t0 = np.zeros(n, np.float32)
    tmax = np.full(n, 3.0, np.float32)
    te, lin, depth, _, _ = [a.cpu().numpy() for a in gpss.eval_local_piece(G, o, d, t0, tmax, np.zeros(n))]
    # (a piece is analytic where mu rises by more than sigma_lo before the cell's exit by
    # the cell's pessimistic edge bound: a minority of starts near a face miss it)
    sel = np.nonzero((lin == 1) & (depth > 1e-6))[0]
    assert len(sel) > n // 8, len(sel)
    assert np.median(depth[sel]) > 1e-2, np.median(depth[sel])
    o, d, t0, tmax, te, depth = o[sel], d[sel], t0[sel], tmax[sel], te[sel], depth[sel]
    m = len(sel)
    # tau grid over [0, depth): collisions t(tau) and the majorant there
    frac = np.linspace(0.0, 1.0, k, endpoint=False)
    tau = (depth[:, None] * frac[None, :]).astype(np.float32)
    rep = lambda a: np.repeat(a, k, axis=0)
    _, _, _, th, sb = [a.cpu().numpy() for a in
                       gpss.eval_local_piece(G, rep(o), rep(d), np.repeat(t0, k), np.repeat(tmax, k), tau.ravel())]
    th, sb = th.reshape(m, k).astype(np.float64), sb.reshape(m, k).astype(np.float64)
    assert np.all(np.diff(th, axis=1) >= 0)
    assert np.all((th >= t0[:, None]) & (th <= te[:, None]))
    # d tau/dt = sbar: the trapezoid integral of the majorant over [t(tau_i), t(tau_j)]
    # gives tau_j - tau_i (the closed-form depth, its inversion and its density agree)
    seg = 0.5 * (sb[:, 1:] + sb[:, :-1]) * np.diff(th, axis=1)
    got = seg.sum(axis=1)
    want = (tau[:, -1] - tau[:, 0]).astype(np.float64)
    rel = np.abs(got - want) / want
    assert np.quantile(rel, 0.95) < 2e-2 and np.median(rel) < 2e-3, (np.median(rel), np.quantile(rel, 0.95))
    # the majorant bounds sigma_t at every sampled point
    pos = (o[:, None, :] + th[..., None].astype(np.float32) * d[:, None, :]).reshape(-1, 3).astype(np.float32)
    st = gpss.eval_sigma_t(G, pos, rep(d)).cpu().numpy().reshape(m, k)
    viol = st > sb * (1 + 1e-6)
    assert not viol.any(), (int(viol.sum()), float((st / sb)[viol].max()))
    # and it is not loose: the expected null collisions of a piece, its majorant's depth
    # minus the true optical depth (trapezoid of sigma_t over the sampled points), stay few
    true_depth = np.sum(0.5 * (st[:, 1:] + st[:, :-1]) * np.diff(th, axis=1), axis=1)
    nulls = tau[:, -1] - true_depth
    assert np.mean(nulls) < 3.0 and np.quantile(nulls, 0.9) < 6.0, (np.mean(nulls), np.quantile(nulls, 0.9))


@pytest.mark.parametrize("lin", [True, False])
def test_ratio_tracking_and_free_flight_unbiased(plane, sphere, lin):
    """Against the oracle's transmittance, with analytic pieces on and off: shadow rays
    through the thin plane ending at the first crossing of mu = 0 (T about 1/2) or
    1.5 sigma/sin(angle) beyond it, and free-flight distances into the thin sphere."""
    sc, G, O = plane
    G.set_surface_flight(lin)
    n = 48
    rng = np.random.default_rng(8)
    ang = np.concatenate([rng.uniform(0.05, 0.3, n // 2), rng.uniform(0.3, 1.4, n - n // 2)])
    phi = rng.uniform(0, 2 * math.pi, n)
    d = np.stack([np.cos(ang) * np.cos(phi), np.cos(ang) * np.sin(phi), -np.sin(ang)], 1).astype(np.float32)
    o = np.stack([rng.uniform(-0.1, 0.1, n), rng.uniform(-0.1, 0.1, n), 0.03 + 0.35 * np.sin(ang)], 1)
    o = o.astype(np.float32)
    sigma = 2.0 ** -10
    tmax = np.zeros(n, np.float32)
    for i in range(n):
        lo, hi = 0.0, 0.7
        for _ in range(50):
            mid = 0.5 * (lo + hi)
            f = oracle.field(O, 0, (o[i] + mid * d[i]).astype(np.float64))
            if f is None or f["mean"] > 0.0:
                lo = mid
            else:
                hi = mid
        tmax[i] = lo + (1.5 * sigma / math.sin(ang[i]) if i % 2 else 0.0)
    ref = np.array([oracle.transmittance(O, o[i].astype(np.float64), d[i].astype(np.float64), float(tmax[i]))
                    for i in range(n)])
    assert ((ref > 0.02) & (ref < 0.98)).mean() > 0.7, ref
    N = 40000
    m = gpss.estimate_transmittance(G, o, d, tmax, N, seed=11).cpu().numpy().astype(np.float64)
    se = np.sqrt(np.maximum(ref * (1 - ref), 1e-4) / N)
    z = (m - ref) / se
    assert np.mean(np.abs(z) > 4) < 0.05, z
    assert abs(np.sum(m - ref)) < 4 * np.sqrt(np.sum(se ** 2))
    sc2, G2, O2 = sphere
    G2.set_surface_flight(lin)
    o1 = np.array([[-0.45, -0.2, 0.35]], np.float32)
    d1 = (np.zeros(3) - o1[0]) / np.linalg.norm(o1[0])
    d1 = d1.astype(np.float32)[None]
    M = 200000
    t = gpss.sample_free_flight(G2, o1, d1, M, seed=5).cpu().numpy()[0]
    for s_ in np.quantile(t[np.isfinite(t)], [0.05, 0.2, 0.5, 0.8, 0.95]):
        p = float(np.mean(t <= s_))
        r = 1 - oracle.transmittance(O2, o1[0].astype(np.float64), d1[0].astype(np.float64), float(s_))
        assert abs(p - r) < 5 * math.sqrt(max(r * (1 - r), 1e-8) / M) + 1e-4, (s_, p, r)
    G.set_surface_flight(True)
    G2.set_surface_flight(True)


def test_images_and_tentative_collisions_against_constant_pieces(sphere):
    sc, G, _ = sphere
    cam = W.perspective_camera(24, 24)
    spp = 2048
    opts = {"spp": spp, "max_bounces": 8, "sampler": "vndf"}  # bounded path weights on both sides
    G.set_surface_flight(True)
    img, sq, sa = gpss.render(G, cam, dict(opts, seed=21), want_sqsum=True)
    G.set_surface_flight(False)
    img2, sq2, sb = gpss.render(G, cam, dict(opts, seed=22), want_sqsum=True)
    G.set_surface_flight(True)
    a, asq = img.cpu().numpy().astype(np.float64), sq.cpu().numpy().astype(np.float64)
    b, bsq = img2.cpu().numpy().astype(np.float64), sq2.cpu().numpy().astype(np.float64)
    z, gm, om, gse, ose = C.image_z(a, asq, spp, b * spp, bsq, spp)
    ok, info = C.check_image_parity(gm, gse, om, ose)
    assert ok, info
    assert sa["aborted"] == 0 and sb["aborted"] == 0
    # tentative collisions (null + shadow steps) per real vertex: no more than with
    # constant pieces (with the projected-area bound a psi(-B/a) both are near the
    # true optical depth on this scene)
    ta = (sa["null_collisions"] + sa["shadow_steps"]) / sa["vertices"]
    tb = (sb["null_collisions"] + sb["shadow_steps"]) / sb["vertices"]
    assert ta <= 1.05 * tb, (ta, tb)
