"""Height-field macrofacets (Sec. 4.1: Beckmann and GGX NDFs about the SDF normal) on
the GPU against the oracle: extinction and phase function to the deterministic bar,
the sampler's weight and pdf, the grid majorant's bound, and images."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_00280_gb300 import gpss
from paper_2603_00280_gb300 import workloads as W
from tests import gpu_common as C
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _scene(kind, length_scale=0.05, n_log2=5):
    sc = C.dyadic_hetero(n_log2, length_scale=length_scale)
    for o in sc["objects"]:
        o["ndf"] = kind
    return sc


@pytest.fixture(scope="module", params=["beckmann", "ggx"])
def hf(request):
    sc = _scene(request.param)
    return request.param, sc, gpss.Scene(sc), oracle.Scene(sc)


def _direction_conditioning(O, x, d, delta=3e-7):
    """Relative change of the oracle's sigma_t when d turns by delta (two orthogonal
    directions): the height-field projected area depends on the angle between d and
    the normal, which FP32 directions and FP32 gradients carry to ~1e-7 rad, and near
    the normal (sigma ~ sin^2) or in the exponential tail of psi that angle is
    ill-conditioned."""
    base = oracle.sigma_t(O, x, d)
    out = np.zeros(len(x))
    for k in range(2):
        t = np.cross(d, np.eye(3)[(np.argmin(np.abs(d), axis=1) + k) % 3])
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        dd = d + delta * t
        dd /= np.linalg.norm(dd, axis=1, keepdims=True)
        out = np.maximum(out, np.abs(oracle.sigma_t(O, x, dd) - base) / np.maximum(base, 1e-300))
    return out


def test_sigma_t_parity(hf):
    kind, sc, G, O = hf
    x = C.dyadic_points(4000, 1)
    d = C.unit_dirs(4000, 2)
    g = gpss.eval_sigma_t(G, x, d).cpu().numpy()
    xd, dd = x.astype(np.float64), d.astype(np.float64)
    o = oracle.sigma_t(O, xd, dd)
    err = C.rel_err(g, o, floor=1e-6 * o.max())
    cond = _direction_conditioning(O, xd, dd)
    assert np.all(err < C.REL + 3.0 * cond), (err.max(), int(np.argmax(err - 3.0 * cond)))
    assert np.quantile(err, 0.99) < C.REL
    assert (o > 1e-3 * o.max()).sum() > 200


def test_phase_function_parity_and_pdf(hf):
    kind, sc, G, O = hf
    n = 2000
    x = C.dyadic_points(n, 3, -0.35, 0.35)
    d = C.unit_dirs(n, 4)
    d2 = C.unit_dirs(n, 5)
    p, pdf = gpss.eval_phase(G, 0, x, d, d2)
    p, pdf = p.cpu().numpy().astype(np.float64), pdf.cpu().numpy().astype(np.float64)
    op, _ = oracle.phase_eval(O, 0, x.astype(np.float64), d.astype(np.float64), d2.astype(np.float64))
    scale = op[:, 0].max()
    err = C.rel_err(p[:, 0], op[:, 0], floor=1e-5 * scale)
    assert err.max() < 1e-4, (err.max(), int(np.argmax(err)))
    assert (op[:, 0] > 1e-3 * scale).sum() > 100
    # pdf: p/F where the ray arrives from above the normal (exact visible normals),
    # the uniform hemisphere's 1/(8 pi |d.m|) otherwise
    for i in np.nonzero(op[:, 0] > 1e-3 * scale)[0][:200]:
        f = oracle.field(O, 0, x[i].astype(np.float64))
        nrm = f["grad"] / np.linalg.norm(f["grad"])
        m = d2[i].astype(np.float64) - d[i]
        m /= np.linalg.norm(m)
        if -d[i] @ nrm > 0:
            want = op[i, 0] / f["albedo"][0]
        else:
            want = 1.0 / (8 * math.pi * abs(d[i] @ m))
        assert pdf[i] == pytest.approx(want, rel=2e-4)


@pytest.mark.parametrize("from_above", [True, False])
def test_sampler_weight_pdf_and_histogram(hf, from_above):
    kind, sc, G, O = hf
    rng = np.random.default_rng(11)
    for _ in range(1000):
        x0 = C.dyadic_points(1, int(rng.integers(1 << 30)), -0.35, 0.35)[0]
        f = oracle.field(O, 0, x0.astype(np.float64))
        if f is not None and abs(f["mean"]) < 0.03:
            break
    nrm = f["grad"] / np.linalg.norm(f["grad"])
    while True:
        d0 = rng.normal(size=3)
        d0 /= np.linalg.norm(d0)
        c = -d0 @ nrm
        if (from_above and c > 0.3) or (not from_above and -0.6 < c < -0.1):
            break
    d0 = d0.astype(np.float32)
    F = f["albedo"][0]
    N = 200000
    u = rng.random((N, 3)).astype(np.float32)
    d2, w, pdf = gpss.sample_phase(G, 0, np.tile(x0, (N, 1)), np.tile(d0, (N, 1)), u)
    d2, w, pdf = d2.cpu().numpy().astype(np.float64), w.cpu().numpy().astype(np.float64), pdf.cpu().numpy()
    ok = w[:, 0] > 0
    # from below the normal the uniform hemisphere about -d also draws half vectors
    # outside the NDF's support (weight 0)
    assert ok.mean() > (0.99 if from_above else 0.05)
    if from_above:
        np.testing.assert_allclose(w[ok, 0], F, rtol=2e-5)  # exact visible normals: weight F
    # E[w] = F (the estimator of the energy through the sampler)
    assert abs(w[:, 0].mean() - F) < 5 * w[:, 0].std() / math.sqrt(N) + 1e-6
    if not from_above:
        return
    # histogram of half vectors about -d against the oracle's p/F
    mh = d2[ok] - d0
    mh /= np.linalg.norm(mh, axis=1, keepdims=True)
    fx, fy, fz = H.frame(-d0.astype(np.float64))
    cz = mh @ fz
    ph = np.mod(np.arctan2(mh @ fy, mh @ fx), 2 * math.pi)
    nb = 8
    cedges = np.quantile(cz, np.linspace(0, 1, nb + 1))
    cedges[0], cedges[-1] = 0.0, 1.0
    obs, _, _ = np.histogram2d(cz, ph, bins=[cedges, np.linspace(0, 2 * math.pi, nb + 1)])
    gx, gw = np.polynomial.legendre.leggauss(16)
    exp_p = np.zeros((nb, nb))
    for i in range(nb):
        c0, c1 = cedges[i], cedges[i + 1]
        cc = 0.5 * (c0 + c1) + 0.5 * (c1 - c0) * gx
        for j in range(nb):
            pp = (j + 0.5 + 0.5 * gx) * 2 * math.pi / nb
            CC, PP = np.meshgrid(cc, pp, indexing="ij")
            WW = np.outer(0.5 * (c1 - c0) * gw, 0.5 * gw * 2 * math.pi / nb).reshape(-1)
            s = np.sqrt(1 - CC ** 2)
            mm = ((s * np.cos(PP))[..., None] * fx + (s * np.sin(PP))[..., None] * fy + CC[..., None] * fz).reshape(-1, 3)
            dd2 = d0 - 2 * (mm @ d0)[:, None] * mm
            pv, _ = oracle.phase_eval(O, 0, np.tile(x0, (len(mm), 1)).astype(np.float64),
                                      np.tile(d0, (len(mm), 1)).astype(np.float64), dd2)
            exp_p[i, j] = np.sum(WW * pv[:, 0] / F * 4 * np.abs(mm @ d0))
    from scipy.stats import chisquare
    assert abs(exp_p.sum() - 1.0) < 5e-3, exp_p.sum()
    # bins outside the visible NDF's support (half vectors below the normal) expect nothing
    empty = exp_p < 1e-12
    assert obs[empty].sum() == 0
    stat, pval = chisquare(obs[~empty], exp_p[~empty] / exp_p[~empty].sum() * obs[~empty].sum())
    assert pval > 1e-4, (stat, pval)


def test_grid_majorant_bounds_sigma_t(hf):
    kind, sc, G, O = hf
    maj = G.majorant().cpu().numpy()
    dims = maj.shape[::-1]
    n = 20000
    x = np.random.default_rng(6).uniform(-0.5, 0.5, size=(n, 3)).astype(np.float32)
    d = C.unit_dirs(n, 7)
    st = gpss.eval_sigma_t(G, x, d).cpu().numpy()
    # majorant grid over the object box [-0.5, 0.5]^3
    idx = np.clip(((x + 0.5) * np.array(dims)).astype(int), 0, np.array(dims) - 1)
    bound = maj[idx[:, 2], idx[:, 1], idx[:, 0]]
    assert np.all(st <= bound * (1 + 1e-6)), float((st / bound).max())


def test_images_match_oracle(hf):
    kind, _, _, _ = hf
    wl = W.heterogeneous(n=32, width=20, height=20, spp=16, max_bounces=10, length_scale=0.05)
    for o in wl["scene"]["objects"]:
        o["ndf"] = kind
    G, O = gpss.Scene(wl["scene"]), oracle.Scene(wl["scene"])
    spp = 8192
    img, sq, st = gpss.render(G, wl["camera"], dict(wl["opts"], spp=spp, seed=3), want_sqsum=True)
    img, sq = img.cpu().numpy().astype(np.float64), sq.cpu().numpy().astype(np.float64)
    s, s2, _ = oracle.render(O, wl["camera"], dict(wl["opts"], spp=128, seed=4, sampler="vndf"))
    z, gm, om, gse, ose = C.image_z(img, sq, spp, s, s2, 128)
    ok, info = C.check_image_parity(gm, gse, om, ose)
    assert ok, info
    assert st["aborted"] == 0


def test_adjoint_rejects_height_fields():
    import torch
    sc = _scene("ggx")
    S = gpss.Scene(sc)
    cam = W.perspective_camera(8, 8)
    g = torch.ones((8, 8, 3), device="cuda")
    with pytest.raises(gpss.GpssError) as e:
        gpss.render_adjoint(S, cam, {"spp": 1, "max_bounces": 2}, g)
    assert e.value.status == 5
