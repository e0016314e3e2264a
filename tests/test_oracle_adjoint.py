"""Pins of the oracle's adjoint (orc_render_grad: path replay of the regular-tracking
estimator with partials from forward-mode dual numbers) against what fixes it
from outside the adjoint:

- every dual partial against central differences of the forward oracle with
  the grid node (or the length scale) perturbed;
- exact single-scatter derivatives on the plane-mean slab (1-D integrals of
  closed forms): slope of the mean, variance, length scale, albedo;
- multi-bounce albedo gradients, exact per path: F does not steer the path, so
  a common-random-number difference of two albedos reproduces every path and
  its chain of vertex factors;
- the scale invariance of the medium, exact per path: (mu, sigma^2) ->
  (c mu, c^2 sigma^2) leaves sigma_t (Eq. generalized_sigma_t) and p (Eq. phase)
  unchanged, so sum(mu dmu + 2 var dvar) = 0;
- multi-bounce mean, variance and length-scale gradients against common-random-
  number differences of the forward oracle (statistical)."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_00280_gb300 import workloads as W
from tests import helpers as H

D45 = np.array([math.cos(math.pi / 4), 0.0, -math.sin(math.pi / 4)])
WL = np.array([0.0, 0.0, 1.0])


def _small_hetero(albedo=0.75, n=16, light=None):
    wl = W.heterogeneous(n=n, width=10, height=10, spp=16, max_bounces=4, length_scale=0.03, albedo=albedo)
    if light is not None:
        wl["scene"]["light"] = light
    return wl


def _scene_with(obj, light, **fields):
    o = dict(obj)
    o.update(fields)
    return oracle.Scene({"objects": [o], "light": light})


@pytest.mark.parametrize("what", ["sigma_t", "projected_area", "ndf", "log_phase"])
def test_dual_partials_match_finite_differences(what):
    """Every derivative slot of the oracle's dual evaluation against a central
    difference of the forward oracle (orc_sigma_t_object, orc_projected_area_world via
    sigma_t/rho, orc_ndf_world and ln p via orc_phase_eval) with one corner
    node's float32 value moved (the actual float32 step is used)."""
    wl = _small_hetero(n=9)
    obj = dict(wl["scene"]["objects"][0])
    # a correlation-scale grid, so its slots are exercised too
    p = W.node_coords((-0.5,) * 3, (0.5,) * 3, (9, 9, 9))
    obj["correlation_scale"] = (1.0 + 0.3 * p[..., 2]).astype(np.float32)
    light = wl["scene"]["light"]
    S = oracle.Scene({"objects": [obj], "light": light})
    rng = np.random.default_rng(7)

    def value(scene, x, d, d2):
        if what == "sigma_t":
            return oracle.sigma_t(scene, x, d)[0]
        f = oracle.field(scene, 0, x)
        if what == "projected_area":
            # sigma(d) = sigma_t / rho with rho = lambda(mu/sigma)/sigma (the oracle's own lambda)
            sig = math.sqrt(f["var"])
            return oracle.sigma_t(scene, x, d)[0] / (oracle.inv_mills(f["mean"] / sig) / sig)
        if what == "ndf":
            # D(m) for the half vector m = d2 here: p(d, reflect(d, m)) / F * 4 sigma(d)
            d_out = d - 2 * np.dot(d, d2) * d2
            pv, _ = oracle.phase_eval(scene, 0, x, d, d_out)
            return pv[0, 0] / f["albedo"][0] * 4 * value_pa(scene, x, d)
        pv, _ = oracle.phase_eval(scene, 0, x, d, d2)
        return math.log(pv[0, 0] / f["albedo"][0])

    def value_pa(scene, x, d):
        f = oracle.field(scene, 0, x)
        sig = math.sqrt(f["var"])
        return oracle.sigma_t(scene, x, d)[0] / (oracle.inv_mills(f["mean"] / sig) / sig)

    checked = 0
    for _ in range(6):
        while True:
            x = rng.uniform(-0.35, 0.35, 3)
            f = oracle.field(S, 0, x)
            if abs(f["mean"]) < 2.5 * math.sqrt(f["var"]):  # in the shell: every slot matters
                break
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        d2 = rng.normal(size=3)
        d2 /= np.linalg.norm(d2)
        if what == "log_phase" or what == "ndf":
            # a half vector that faces the arriving ray, away from the NDF's underflow
            g = f["grad"] / np.linalg.norm(f["grad"])
            m = g + 0.3 * rng.normal(size=3)
            m /= np.linalg.norm(m)
            if np.dot(d, m) > 0:
                d = -d
            # log_phase takes the outgoing direction, ndf the half vector itself
            d2 = d - 2 * np.dot(d, m) * m if what == "log_phase" else m
        r = oracle.dual_eval(S, 0, what, x, d, d2)
        assert r is not None
        v0, der, node = r
        # the dual's value against the forward oracle (for D: its own quadrature)
        assert v0 == pytest.approx(value(S, x, d, d2), rel=1e-9, abs=1e-14)
        scale = max(abs(der).max(), 1e-300)
        for base, field in ((oracle.SLOT_MEAN, "mean"), (oracle.SLOT_VAR, "var"), (oracle.SLOT_CS, "correlation_scale")):
            for k in range(8):
                nd = int(node[k])
                grid = np.ascontiguousarray(obj[field], dtype=np.float32)
                v = float(grid.reshape(-1)[nd])
                h = 1e-3 * max(abs(v), 1e-3)
                up, dn = grid.copy(), grid.copy()
                up.reshape(-1)[nd] = np.float32(v + h)
                dn.reshape(-1)[nd] = np.float32(v - h)
                hh = float(up.reshape(-1)[nd]) - float(dn.reshape(-1)[nd])
                fd = (value(_scene_with(obj, light, **{field: up}), x, d, d2)
                      - value(_scene_with(obj, light, **{field: dn}), x, d, d2)) / hh
                assert der[base + k] == pytest.approx(fd, rel=2e-5, abs=2e-6 * scale), (field, k, der[base + k], fd)
                checked += 1
        l = obj["length_scale"]
        fd = (value(_scene_with(obj, light, length_scale=l * (1 + 1e-5)), x, d, d2)
              - value(_scene_with(obj, light, length_scale=l * (1 - 1e-5)), x, d, d2)) / (2e-5 * l)
        assert der[oracle.SLOT_L] == pytest.approx(fd, rel=2e-5, abs=2e-6 * scale)
        # the albedo does not enter these quantities
        assert np.all(der[oracle.SLOT_ALB:oracle.SLOT_ALB + 8] == 0.0)
    assert checked == 6 * 24


def _batches(scene, cam, opts, d_image, seeds, **kw):
    return [oracle.render_grad(scene, cam, dict(opts, seed=s), d_image, **kw) for s in seeds]


def test_single_scatter_gradients_are_exact():
    """max_bounces = 1 on the plane-mean slab lit from +z, seen at 45 degrees: every
    interior pixel is a 1-D integral of closed forms (the plane's transmittance both
    ways, a constant phase function), so its derivatives with respect to the slope of
    the mean (mu = c z), the variance, the length scale and the albedo are exact."""
    F = 0.75
    S = oracle.Scene(H.dyadic_slab(albedo=F))
    cam = W.ortho_camera_45(16, 16, film=0.5)
    g = np.zeros((16, 16, 3))
    g[6:10, 6:10, :] = 1.0
    npx = 16 * 3
    z = W.node_coords(H.SLAB_BMIN, H.SLAB_BMAX, (17, 17, 9))[..., 2].reshape(-1)
    rows = []
    for r, st in _batches(S, cam, {"spp": 128, "max_bounces": 1}, g, range(100, 108), rows=(6, 10, 1), cols=(6, 10)):
        assert st["mismatch"] == 0
        r = r[0]
        rows.append([(r["mean"] * z).sum(), r["var"].sum(), r["l"], r["albedo"].sum()])
    e = np.array(rows) / npx
    m, se = e.mean(0), e.std(0, ddof=1) / math.sqrt(len(e))
    sig, l = H.SLAB_SIGMA, H.SLAB_L
    h = 1e-4
    f = lambda **kw: H.slab_single_scatter(D45, WL, F, **kw)
    exact = [
        (f(slope=1 + h) - f(slope=1 - h)) / (2 * h),
        (f(sigma=sig * math.sqrt(1 + h)) - f(sigma=sig * math.sqrt(1 - h))) / (2 * h * sig * sig),
        (f(l=l * (1 + h)) - f(l=l * (1 - h))) / (2 * h * l),
        f() / F,
    ]
    for name, mm, ss, ex in zip(("slope", "variance", "l", "albedo"), m, se, exact):
        assert abs(mm - ex) < 4 * ss + 1e-6 * abs(ex), (name, mm, ss, ex)
        assert ss < 0.03 * abs(ex), (name, ss, ex)  # the test has power


def test_multibounce_albedo_gradient_is_exact_per_path():
    """The albedo scales the phase function but steers nothing (the sampling mixture
    and the free flights do not depend on F), so with common random numbers a
    difference of two uniform albedos retraces every path: the summed albedo
    gradient (F times d/dF of the image) equals that difference to its O(h^2)
    truncation.  This pins which radiance every vertex factor is weighted with
    (the vertex's NEE contribution, and everything collected after it)."""
    F = 0.75
    eps = 2.0 ** -10  # F (1 +- eps) is exact in float32
    wl = _small_hetero(albedo=F)
    sc, cam = wl["scene"], wl["camera"]
    obj = sc["objects"][0]
    S = oracle.Scene(sc)
    g = np.zeros((10, 10, 3))
    g[..., 0] = 1.0
    g[..., 2] = 0.5
    opts = dict(wl["opts"], spp=16, seed=10)
    (r,), st = oracle.render_grad(S, cam, opts, g, want=("albedo",))
    adj = r["albedo"].sum() * F
    Sp = _scene_with(obj, sc["light"], albedo=np.float32(F * (1 + eps)) * np.ones_like(obj["albedo"]))
    Sm = _scene_with(obj, sc["light"], albedo=np.float32(F * (1 - eps)) * np.ones_like(obj["albedo"]))
    s, _, _ = oracle.render_diff(Sp, Sm, cam, opts)
    fd = (s * g).sum() / opts["spp"] / (2 * eps)
    assert st["vertices"] > 500
    assert adj == pytest.approx(fd, rel=2e-5)


def test_scale_invariance_of_the_medium_holds_per_path():
    """(mu, sigma^2) -> (c mu, c^2 sigma^2) maps rho to rho/c and sigma(d), D(m) to c
    times themselves, so sigma_t and p are unchanged and so is every path: the
    adjoint's sum(mu dL/dmu + 2 var dL/dvar) vanishes (to rounding), which ties the
    mean-gradient, mean-value and variance partials together on every node."""
    wl = _small_hetero()
    sc, cam = wl["scene"], wl["camera"]
    obj = sc["objects"][0]
    S = oracle.Scene(sc)
    g = np.ones((10, 10, 3))
    (r,), st = oracle.render_grad(S, cam, dict(wl["opts"], spp=8, seed=3), g, want=("mean", "var"))
    mu = np.asarray(obj["mean"], np.float64).reshape(-1)
    var = np.asarray(obj["var"], np.float64).reshape(-1)
    a, b = (mu * r["mean"]).sum(), 2 * (var * r["var"]).sum()
    assert abs(a) > 1.0  # both parts are large ...
    assert abs(a + b) < 1e-6 * (abs(a) + abs(b))  # ... and cancel


def test_multibounce_gradients_match_crn_finite_differences():
    """Multi-bounce plane-mean slab (4 bounces, about 3 real vertices per path,
    directional light): d/dl, d/d(slope of the mean) and d/d(variance) of the
    interior pixels against central differences of the forward oracle with common
    random numbers.  Both estimate the same derivative of the expected image; the
    differences include every bounce's phase-sample factor and flight (statistical
    pin, about 5% power)."""
    sc = H.dyadic_slab(albedo=0.75)
    obj = sc["objects"][0]
    S = oracle.Scene(sc)
    cam = W.ortho_camera_45(16, 16, film=0.5)
    opts = {"spp": 64, "max_bounces": 4}
    win = dict(rows=(6, 10, 1), cols=(6, 10))
    g = np.zeros((16, 16, 3))
    g[6:10, 6:10, 0] = 1.0
    z = W.node_coords(H.SLAB_BMIN, H.SLAB_BMAX, (17, 17, 9))[..., 2]
    rows = []
    for (r,), st in _batches(S, cam, opts, g, range(20, 28), want=("mean", "var", "l"), **win):
        assert st["mismatch"] == 0
        rows.append([r["l"], (r["mean"] * z.reshape(-1)).sum(), r["var"].sum()])
    e = np.array(rows)
    m, se = e.mean(0), e.std(0, ddof=1) / math.sqrt(len(e))

    def fd(h, seed, **fields_pm):
        up = {k: v[0] for k, v in fields_pm.items()}
        dn = {k: v[1] for k, v in fields_pm.items()}
        spp = 1024
        s, s2, _ = oracle.render_diff(_scene_with(obj, sc["light"], **up), _scene_with(obj, sc["light"], **dn), cam,
                                      dict(opts, spp=spp, seed=seed), **win)
        v = s[..., 0].sum() / spp / h
        return v, math.sqrt(max(np.sum(s2[..., 0] / spp - (s[..., 0] / spp) ** 2), 0) / spp) / h

    eps = 2.0 ** -5  # the perturbed grids are exact in float32
    l = obj["length_scale"]
    v0 = float(obj["var"].reshape(-1)[0])
    fds = [
        fd(2 * eps * l, 5, length_scale=(l * (1 + eps), l * (1 - eps))),
        fd(2 * eps, 6, mean=((z * (1 + eps)).astype(np.float32), (z * (1 - eps)).astype(np.float32))),
        fd(2 * eps * v0, 7, var=(np.full_like(obj["var"], v0 * (1 + eps)), np.full_like(obj["var"], v0 * (1 - eps)))),
    ]
    for name, mm, ss, (fv, fse) in zip(("l", "slope", "variance"), m, se, fds):
        assert abs(mm - fv) < 4 * math.sqrt(ss * ss + fse * fse) + 0.01 * abs(fv), (name, mm, ss, fv, fse)
        assert ss < 0.05 * abs(mm), (name, ss, mm)  # the test has power


def test_adjoint_rejects_what_it_does_not_support():
    wl = _small_hetero(n=9)
    obj = dict(wl["scene"]["objects"][0])
    obj["length_scale_n"] = 0.5 * obj["length_scale"]
    S = oracle.Scene({"objects": [obj], "light": wl["scene"]["light"]})
    with pytest.raises(NotImplementedError):
        oracle.render_grad(S, wl["camera"], wl["opts"], np.ones((10, 10, 3)))
