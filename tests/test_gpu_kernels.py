"""Anisotropic and non-stationary kernels (gradient covariance sigma^2 diag(1/l_t^2,
1/l_b^2, 1/l_n^2) in the frame of a tangent field and the mean gradient, every l scaled
by a correlation-scale grid) on the GPU against the FP64 oracle: extinction and phase
function to the deterministic bar (plus the FP32 conditioning of the directions), both
samplers' weights, pdfs and histograms, the grid and local majorants' bounds, images,
and the adjoint's gradient with respect to the correlation-scale grid."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_00280_gb300 import gpss
from paper_2603_00280_gb300 import workloads as W
from tests import gpu_common as C
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _kernel_scene(length_scale=0.05, n_log2=5, **kw):
    sc = C.dyadic_hetero(n_log2, length_scale=length_scale)
    sc["objects"] = [W.with_kernel(sc["objects"][0], **kw)]
    return sc


@pytest.fixture(scope="module")
def kern():
    sc = _kernel_scene()
    return sc, gpss.Scene(sc), oracle.Scene(sc)


def _rotations(d, delta):
    """d turned by delta about two axes orthogonal to it (FP64, renormalised)."""
    out = []
    for k in range(2):
        t = np.cross(d, np.eye(3)[(np.argmin(np.abs(d), axis=1) + k) % 3])
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        dd = d + delta * t
        out.append(dd / np.linalg.norm(dd, axis=1, keepdims=True))
    return out


def _conditioning(fn, d, d2=None, delta=3e-7):
    """Largest relative change of fn(d[, d2]) when a direction turns by delta: FP32
    directions and interpolated gradients carry ~1e-7 rad, which the exponential
    tails of the projected area and of the NDF amplify."""
    base = fn(d) if d2 is None else fn(d, d2)
    out = np.zeros(len(d))
    for dd in _rotations(d, delta):
        v = fn(dd) if d2 is None else fn(dd, d2)
        out = np.maximum(out, np.abs(v - base) / np.maximum(np.abs(base), 1e-300))
    if d2 is not None:
        for dd in _rotations(d2, delta):
            v = fn(d, dd)
            out = np.maximum(out, np.abs(v - base) / np.maximum(np.abs(base), 1e-300))
    return out


def test_sigma_t_parity(kern):
    sc, G, O = kern
    x = C.dyadic_points(4000, 1)
    d = C.unit_dirs(4000, 2)
    g = gpss.eval_sigma_t(G, x, d).cpu().numpy()
    xd, dd = x.astype(np.float64), d.astype(np.float64)
    o = oracle.sigma_t(O, xd, dd)
    err = C.rel_err(g, o, floor=1e-6 * o.max())
    cond = _conditioning(lambda v: oracle.sigma_t(O, xd, v), dd)
    assert np.all(err < C.REL + 3.0 * cond), (err.max(), int(np.argmax(err - 3.0 * cond)))
    assert np.quantile(err, 0.99) < C.REL
    assert (o > 1e-3 * o.max()).sum() > 200


def test_phase_function_and_mixture_pdf_parity(kern):
    sc, G, O = kern
    n = 1500
    x = C.dyadic_points(n, 3, -0.35, 0.35)
    d = C.unit_dirs(n, 4)
    d2 = C.unit_dirs(n, 5)
    xd, dd, d2d = x.astype(np.float64), d.astype(np.float64), d2.astype(np.float64)
    for R in (0.5, 0.2):
        p, pdf = gpss.eval_phase(G, 0, x, d, d2, R)
        p, pdf = p.cpu().numpy()[:, 0].astype(np.float64), pdf.cpu().numpy().astype(np.float64)
        op, opdf = oracle.phase_eval(O, 0, xd, dd, d2d, R)
        cp = _conditioning(lambda a, b: oracle.phase_eval(O, 0, xd, a, b, R)[0][:, 0], dd, d2d)
        cq = _conditioning(lambda a, b: oracle.phase_eval(O, 0, xd, a, b, R)[1], dd, d2d)
        e1 = C.rel_err(p, op[:, 0], floor=1e-6 * op[:, 0].max())
        e2 = C.rel_err(pdf, opdf, floor=1e-6 * opdf.max())
        # the closed-form anisotropic NDF (FP32 moments) against the oracle's quadrature
        assert np.all(e1 < 1e-4 + 3.0 * cp), (e1.max(), int(np.argmax(e1 - 3 * cp)))
        assert np.quantile(e1, 0.99) < 2e-5
        assert np.all(e2 < C.REL + 4.0 * cq), (e2.max(), int(np.argmax(e2 - 4 * cq)))
        assert (op[:, 0] > 1e-3 * op[:, 0].max()).sum() > 100


def _shell_point(O, seed, beta_sign):
    rng = np.random.default_rng(seed)
    for _ in range(2000):
        x = C.dyadic_points(1, int(rng.integers(1 << 30)), -0.35, 0.35)[0]
        f = oracle.field(O, 0, x.astype(np.float64))
        if f is None or abs(f["mean"]) > 0.03:
            continue
        g = f["grad"] / np.linalg.norm(f["grad"])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        c = -d @ g
        if (beta_sign > 0 and c > 0.3) or (beta_sign < 0 and -0.4 < c < -0.05):
            return x, d.astype(np.float32), f
    raise RuntimeError("no configuration found")


def _histogram_check(O, x0, d0, d2, F, nb=8):
    """chi^2 of half vectors about -d0 on (cos, azimuth) bins against the oracle's p/F."""
    from scipy.stats import chisquare
    mh = d2 - d0
    mh /= np.linalg.norm(mh, axis=1, keepdims=True)
    fx, fy, fz = H.frame(-d0.astype(np.float64))
    cz = mh @ fz
    ph = np.mod(np.arctan2(mh @ fy, mh @ fx), 2 * math.pi)
    cedges = np.quantile(cz, np.linspace(0, 1, nb + 1))
    cedges[0], cedges[-1] = 0.0, 1.0
    obs, _, _ = np.histogram2d(cz, ph, bins=[cedges, np.linspace(0, 2 * math.pi, nb + 1)])
    gx, gw = np.polynomial.legendre.leggauss(12)
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
    assert abs(exp_p.sum() - 1.0) < 5e-3, exp_p.sum()
    stat, pval = chisquare(obs.ravel(), exp_p.ravel() / exp_p.sum() * obs.sum())
    assert pval > 1e-4, (stat, pval)


@pytest.mark.parametrize("beta_sign", [1, -1])
def test_exact_vndf_sampler(kern, beta_sign):
    """The exact visible-normal sampler with the anisotropic covariance: weight F,
    pdf = p/F at the sampled direction, histogram of p/F."""
    sc, G, O = kern
    x0, d0, f = _shell_point(O, 40 + beta_sign, beta_sign)
    n = 200000
    u = np.random.default_rng(31).random((n, 3)).astype(np.float32)
    xs, ds = np.tile(x0, (n, 1)), np.tile(d0, (n, 1))
    d2, w, pdf = gpss.sample_phase_vndf(G, 0, xs, ds, u)
    d2, w, pdf = d2.cpu().numpy().astype(np.float64), w.cpu().numpy(), pdf.cpu().numpy().astype(np.float64)
    F = f["albedo"][0]
    assert np.all(pdf > 0)
    np.testing.assert_allclose(w[:, 0], F, rtol=1e-6)
    mh = d2 - d0
    mh /= np.linalg.norm(mh, axis=1, keepdims=True)
    keep = np.nonzero(np.abs(mh @ d0) > 0.05)[0][:200]
    op, _ = oracle.phase_eval(O, 0, xs[keep].astype(np.float64), ds[keep].astype(np.float64), d2[keep])
    np.testing.assert_allclose(pdf[keep], op[:, 0] / F, rtol=5e-4)
    _histogram_check(O, x0, d0, d2, F)


def test_mixture_sampler_weight_and_pdf(kern):
    sc, G, O = kern
    x0, d0, f = _shell_point(O, 44, 1)
    n = 100000
    u = np.random.default_rng(32).random((n, 3)).astype(np.float32)
    xs, ds = np.tile(x0, (n, 1)), np.tile(d0, (n, 1))
    d2, w, pdf = gpss.sample_phase(G, 0, xs, ds, u)
    d2, w, pdf = d2.cpu().numpy().astype(np.float64), w.cpu().numpy(), pdf.cpu().numpy()
    mh = d2 - d0
    mh /= np.linalg.norm(mh, axis=1, keepdims=True)
    keep = np.nonzero((np.abs(mh @ d0) > 0.05) & (w[:, 0] > 0))[0][:300]
    op, opdf = oracle.phase_eval(O, 0, xs[keep].astype(np.float64), ds[keep].astype(np.float64), d2[keep])
    np.testing.assert_allclose(pdf[keep], opdf, rtol=2e-4)
    np.testing.assert_allclose(w[keep, 0], op[:, 0] / opdf, rtol=5e-4)
    F = f["albedo"][0]
    assert abs(w[:, 0].mean() - F) < 5 * w[:, 0].std() / math.sqrt(n)


def test_grid_majorant_bounds_sigma_t(kern):
    sc, G, O = kern
    maj = G.majorant().cpu().numpy()
    dims = maj.shape[::-1]
    n = 20000
    x = np.random.default_rng(6).uniform(-0.5, 0.5, size=(n, 3)).astype(np.float32)
    d = C.unit_dirs(n, 7)
    st = gpss.eval_sigma_t(G, x, d).cpu().numpy()
    idx = np.clip(((x + 0.5) * np.array(dims)).astype(int), 0, np.array(dims) - 1)
    bound = maj[idx[:, 2], idx[:, 1], idx[:, 0]]
    assert np.all(st <= bound * (1 + 1e-6)), float((st / bound).max())


def test_local_majorant_bounds_sigma_t():
    """A thin shell (sigma = 2^-10, spacing 1/16) with the anisotropic non-stationary
    kernel: every local-majorant piece bounds sigma_t on [t0, t_end)."""
    p = W.node_coords((-0.5,) * 3, (0.5,) * 3, (17, 17, 17))
    mean = p[..., 2] - 0.03 + 0.02 * W.value_noise_grid((-0.5,) * 3, (0.5,) * 3, (17, 17, 17), 11)
    obj = W.with_kernel(W.make_object(mean, 2.0 ** -20, 0.8, (-0.5,) * 3, (0.5,) * 3, 0.01))
    G = gpss.Scene({"objects": [obj], "light": W.sky_light()})
    n, k = 4096, 97
    rng = np.random.default_rng(3)
    o = rng.uniform(-0.49, 0.49, size=(n, 3)).astype(np.float32)
    o[:, 2] = rng.uniform(-0.1, 0.15, size=n)
    d = C.unit_dirs(n, 4)
    d[: n // 4, 2] *= 0.02
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t0 = np.zeros(n, np.float32)
    tmax = np.full(n, 2.0, np.float32)
    te, sb = gpss.eval_local_majorant(G, o, d, t0, tmax)
    te, sb = te.cpu().numpy(), sb.cpu().numpy()
    s = np.linspace(0.0, 1.0 - 1e-4, k)
    t = t0[:, None] + (np.maximum(te, t0) - t0)[:, None] * s[None, :]
    pos = (o[:, None, :] + t[..., None] * d[:, None, :]).reshape(-1, 3).astype(np.float32)
    st = gpss.eval_sigma_t(G, pos, np.repeat(d, k, axis=0)).cpu().numpy().reshape(n, k)
    ok = te > t0
    assert ok.mean() > 0.99
    viol = (st > sb[:, None]) & ok[:, None]
    assert not viol.any(), (int(viol.sum()), float((st / sb[:, None])[viol].max()))


@pytest.mark.parametrize("sampler", ["mixture", "vndf"])
def test_images_match_oracle(sampler):
    wl = W.nonstationary(n=32, width=20, height=20, spp=16, max_bounces=10, length_scale=0.05)
    G, O = gpss.Scene(wl["scene"]), oracle.Scene(wl["scene"])
    spp = 8192
    opts = dict(wl["opts"], spp=spp, seed=3, sampler=sampler)
    img, sq, st = gpss.render(G, wl["camera"], opts, want_sqsum=True)
    img, sq = img.cpu().numpy().astype(np.float64), sq.cpu().numpy().astype(np.float64)
    s, s2, _ = oracle.render(O, wl["camera"], dict(wl["opts"], spp=128, seed=4, sampler="vndf"))
    z, gm, om, gse, ose = C.image_z(img, sq, spp, s, s2, 128)
    ok, info = C.check_image_parity(gm, gse, om, ose)
    assert ok, info
    assert st["aborted"] == 0


def test_batch_with_kernels_equals_separate_renders():
    js = [W.nonstationary(n=24, width=24, height=24, spp=8, max_bounces=6, seed=s) for s in range(2)]
    js.append(W.heterogeneous(n=24, width=24, height=24, spp=8, max_bounces=6, seed=9))
    scenes = [gpss.Scene(j["scene"]) for j in js]
    ref = [gpss.render(S, j["camera"], j["opts"])[0].cpu().numpy() for S, j in zip(scenes, js)]
    with gpss.Batch(scenes, [j["camera"] for j in js], [j["opts"] for j in js], block_size=128) as B:
        imgs, _, _ = B.render()
    # the two kernels may round a rare decision differently (approximate FP32 division):
    # all but 1% of the pixels agree to the film's float-summation order, totals to 1e-3
    for x, y in zip(imgs, ref):
        x = x.cpu().numpy().astype(np.float64)
        y = y.astype(np.float64)
        bad = np.abs(x - y) > 1e-6 + 2e-5 * np.maximum(np.abs(x), np.abs(y))
        assert bad.mean() <= 0.01, int(bad.sum())
        assert abs(x.sum() - y.sum()) <= 1e-3 * abs(y.sum())


# ----------------------------------------------------------------- adjoint
def _cs_scene():
    """Isotropic kernel with a correlation-scale ramp (the adjoint's supported case)."""
    wl = W.heterogeneous(n=16, width=10, height=10, spp=64, max_bounces=4, length_scale=0.03)
    obj = W.with_kernel(wl["scene"]["objects"][0], l_b_ratio=1.0, l_n_ratio=1.0, tangent=False)
    wl["scene"]["objects"] = [obj]
    return wl


def _cs_direction(obj):
    """A smooth perturbation direction of the correlation-scale grid."""
    p = W.node_coords(obj["bbox_min"], obj["bbox_max"], obj["mean"].shape[::-1])
    return (0.5 + 0.5 * p[..., 0] - 0.3 * p[..., 1]).astype(np.float64)


def _adjoint_cs(wl, seeds, spp):
    import torch
    sc, cam = wl["scene"], wl["camera"]
    obj = sc["objects"][0]
    S = gpss.Scene(sc)
    g = torch.zeros((cam["height"], cam["width"], 3), device="cuda")
    g[..., 0] = 1.0
    out_cs, out_l = [], []
    for sd in seeds:
        dc = torch.zeros(obj["mean"].shape, device="cuda")
        dl = torch.zeros(1, device="cuda")
        st = gpss.render_adjoint(S, cam, dict(wl["opts"], spp=spp, seed=sd), g, None, None, None, dl, dc)
        assert st["aborted"] == 0
        out_cs.append(dc.cpu().numpy().astype(np.float64))
        out_l.append(float(dl[0]))
    return out_cs, np.array(out_l)


def _mse(a):
    a = np.asarray(a, np.float64)
    return a.mean(), a.std(ddof=1) / math.sqrt(len(a))


def test_correlation_scale_gradient_against_oracle_finite_differences():
    wl = _cs_scene()
    sc, cam = wl["scene"], wl["camera"]
    obj = sc["objects"][0]
    v = _cs_direction(obj)
    dcs, _ = _adjoint_cs(wl, range(11, 19), 4096)
    eps = 0.02
    op = dict(obj, correlation_scale=(obj["correlation_scale"] * (1 + eps * v)).astype(np.float32))
    om = dict(obj, correlation_scale=(obj["correlation_scale"] * (1 - eps * v)).astype(np.float32))
    # the direction in s-space actually taken (the FP32 grids as stored)
    step = (op["correlation_scale"].astype(np.float64) - om["correlation_scale"].astype(np.float64))
    adj = [(dc * step).sum() for dc in dcs]
    a, ase = _mse(adj)
    Sp = oracle.Scene({"objects": [op], "light": sc["light"]})
    Sm = oracle.Scene({"objects": [om], "light": sc["light"]})
    ospp = 384
    s, s2, _ = oracle.render_diff(Sp, Sm, cam, dict(wl["opts"], spp=ospp, seed=6))
    fd = s[..., 0].sum() / ospp
    fd_se = math.sqrt(max(np.sum(s2[..., 0] / ospp - (s[..., 0] / ospp) ** 2), 0) / ospp)
    assert abs(a) > 3 * ase, (a, ase)
    assert abs(a - fd) < 4 * math.sqrt(ase ** 2 + fd_se ** 2) + 0.03 * abs(fd), (a, ase, fd, fd_se)


def test_correlation_scale_and_length_scale_gradients_against_gpu_finite_differences():
    wl = _cs_scene()
    sc, cam = wl["scene"], wl["camera"]
    obj = sc["objects"][0]
    v = _cs_direction(obj)
    seeds = list(range(21, 29))
    dcs, dls = _adjoint_cs(wl, seeds, 4096)
    eps = 0.01
    fd_cs, fd_l = [], []
    for sd in seeds:
        vals = []
        for sign in (1, -1):
            o = dict(obj, correlation_scale=(obj["correlation_scale"] * (1 + sign * eps * v)).astype(np.float32))
            img, _, _ = gpss.render(gpss.Scene({"objects": [o], "light": sc["light"]}), cam,
                                    dict(wl["opts"], spp=4096, seed=sd))
            vals.append(float(img[..., 0].double().sum()))
        fd_cs.append((vals[0] - vals[1]))
        vals = []
        for sign in (1, -1):
            o = dict(obj, length_scale=obj["length_scale"] * (1 + sign * eps))
            img, _, _ = gpss.render(gpss.Scene({"objects": [o], "light": sc["light"]}), cam,
                                    dict(wl["opts"], spp=4096, seed=sd))
            vals.append(float(img[..., 0].double().sum()))
        fd_l.append((vals[0] - vals[1]) / (2 * eps * obj["length_scale"]))
    step = (obj["correlation_scale"] * (1 + eps * v)).astype(np.float32).astype(np.float64) - \
           (obj["correlation_scale"] * (1 - eps * v)).astype(np.float32).astype(np.float64)
    adj_cs = [(dc * step).sum() for dc in dcs]
    for name, fd, adj in (("correlation scale", fd_cs, adj_cs), ("l", fd_l, dls)):
        a, ase = _mse(adj)
        f, fse = _mse(fd)
        assert abs(a) > 3 * ase, (name, a, ase)
        assert abs(a - f) < 4 * math.sqrt(ase ** 2 + fse ** 2) + 0.03 * abs(f), (name, a, ase, f, fse)


def test_adjoint_kernel_edge_cases():
    import torch
    wl = _cs_scene()
    sc, cam = wl["scene"], wl["camera"]
    obj = sc["objects"][0]
    g = torch.ones((10, 10, 3), device="cuda")
    # anisotropic kernels are not differentiable here
    for kw in ({"l_b_ratio": 2.0}, {"l_n_ratio": 0.5, "tangent": False}):
        o = W.with_kernel(W.heterogeneous(n=16, length_scale=0.03)["scene"]["objects"][0], **kw)
        with pytest.raises(gpss.GpssError) as e:
            gpss.render_adjoint(gpss.Scene({"objects": [o], "light": sc["light"]}), cam, wl["opts"], g)
        assert e.value.status == 5
    # a correlation-scale gradient for an object without the grid is an argument error
    plain = W.heterogeneous(n=16, width=10, height=10, length_scale=0.03)
    dc = torch.zeros(obj["mean"].shape, device="cuda")
    with pytest.raises(gpss.GpssError) as e:
        gpss.render_adjoint(gpss.Scene(plain["scene"]), cam, wl["opts"], g, None, None, None, None, dc)
    assert e.value.status == 1
    # autograd through render_differentiable with a correlation-scale tensor
    S = gpss.Scene(sc)
    mean = torch.tensor(obj["mean"], device="cuda", requires_grad=True)
    var = torch.tensor(obj["var"], device="cuda", requires_grad=True)
    alb = torch.tensor(obj["albedo"], device="cuda", requires_grad=True)
    l = torch.tensor(obj["length_scale"], device="cuda", requires_grad=True)
    cs = torch.tensor(obj["correlation_scale"], device="cuda", requires_grad=True)
    img = gpss.render_differentiable(S, obj, mean, var, alb, l, cam, dict(wl["opts"], spp=16),
                                     correlation_scale=cs)
    (img ** 2).sum().backward()
    assert cs.grad is not None and torch.isfinite(cs.grad).all() and float(cs.grad.abs().sum()) > 0
    assert torch.isfinite(mean.grad).all() and float(l.grad.abs()) > 0


def test_scene_validation_of_kernels():
    base = W.heterogeneous(n=16, length_scale=0.03)["scene"]
    obj = base["objects"][0]
    bad = [
        dict(obj, length_scale_b=0.06),  # l_b != l_t without a tangent field
        dict(obj, correlation_scale=np.zeros(obj["mean"].shape, np.float32)),
        dict(W.with_kernel(obj), tangent=np.full((3,) + obj["mean"].shape, np.nan, np.float32)),
        dict(obj, ndf="ggx", length_scale_n=0.06),  # height fields take an isotropic kernel
        dict(obj, length_scale_n=-1.0),
    ]
    for o in bad:
        with pytest.raises(gpss.GpssError) as e:
            gpss.Scene({"objects": [o], "light": base["light"]})
        assert e.value.status == 1
    # updates may add and drop the kernel grids
    S = gpss.Scene(base)
    S.update([W.with_kernel(obj)])
    x = C.dyadic_points(64, 1)
    d = C.unit_dirs(64, 2)
    a = gpss.eval_sigma_t(S, x, d).cpu().numpy()
    b = gpss.eval_sigma_t(gpss.Scene({"objects": [W.with_kernel(obj)], "light": base["light"]}), x, d).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    S.update([obj])
    c = gpss.eval_sigma_t(S, x, d).cpu().numpy()
    np.testing.assert_array_equal(c, gpss.eval_sigma_t(gpss.Scene(base), x, d).cpu().numpy())
