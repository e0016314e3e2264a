"""Pins of the oracle's fields, projected area and NDF (Sec. 4 of the paper).

Each check compares the oracle with something other than itself: scipy
quadrature of the defining integral, the paper's printed closed form, exact
sphere-integral identities, textbook Beckmann limits, or exact interpolation.
"""
import math

import numpy as np
import pytest
import scipy.special as sp
from scipy.integrate import quad

import oracle
from paper_2603_00280_gb300 import workloads as W
from tests import helpers as H



# ------------------------------------------------------------- fields
def test_trilinear_reproduces_linear_fields_and_gradient():
    bmin, bmax = np.array([-0.3, 0.1, -1.0]), np.array([0.5, 0.9, 0.2])
    n = (5, 7, 4)
    p = W.node_coords(bmin, bmax, n)
    a, b = np.array([0.25, -0.5, 2.0]), 0.125
    mean = p @ a + b
    var = np.full(mean.shape, 0.01)
    obj = W.make_object(mean, var, 0.5, bmin, bmax, 0.1)
    S = oracle.Scene({"objects": [obj], "light": W.sky_light()})
    RNG = np.random.default_rng(10)
    for _ in range(50):
        x = bmin + RNG.random(3) * (bmax - bmin)
        f = oracle.field(S, 0, x)
        assert f["mean"] == pytest.approx(float(np.float64(np.float32(1)) * (x @ a + b)), abs=2e-6)
        np.testing.assert_allclose(f["grad"], a, atol=2e-5)
        assert f["var"] == pytest.approx(0.01, rel=1e-6)
    assert oracle.field(S, 0, bmax + 1e-9) is None
    assert oracle.field(S, 0, bmin) is not None and oracle.field(S, 0, bmax) is not None


def test_trilinear_is_exact_at_nodes_and_continuous_across_faces():
    bmin, bmax = np.zeros(3), np.ones(3)
    n = (4, 4, 4)
    RNG = np.random.default_rng(11)
    vals = RNG.random((4, 4, 4)).astype(np.float32)
    obj = W.make_object(vals, 0.02, 0.5, bmin, bmax, 0.1)
    S = oracle.Scene({"objects": [obj], "light": W.sky_light()})
    for (i, j, k) in [(0, 0, 0), (1, 2, 3), (3, 3, 3), (2, 0, 1)]:
        x = np.array([i, j, k]) / 3.0
        assert oracle.field(S, 0, x)["mean"] == pytest.approx(float(vals[k, j, i]), abs=1e-12)
    x = np.array([1 / 3.0, 0.4, 0.7])
    lo = oracle.field(S, 0, x - [1e-12, 0, 0])["mean"]
    hi = oracle.field(S, 0, x + [1e-12, 0, 0])["mean"]
    assert lo == pytest.approx(hi, abs=1e-9)


# ------------------------------------------------------------- projected area sigma(w)
def _rand_params(n, seed):
    RNG = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        w = RNG.normal(size=3)
        w /= np.linalg.norm(w)
        ax, ay, az = np.exp(RNG.uniform(math.log(0.05), math.log(5.0), 3))
        G = RNG.uniform(0.0, 2.0)
        out.append((w, G, ax, ay, az))
    return out


@pytest.mark.parametrize("w,G,ax,ay,az", _rand_params(25, 1))
def test_projected_area_equals_gaussian_expectation(w, G, ax, ay, az):
    """Eq. generalized_lambda times cos == E[max(0,-w.g)] (the definition, by quadrature)."""
    ref = H.projected_area_by_quadrature(w, G, ax, ay, az)
    assert oracle.projected_area_local(w, G, ax, ay, az) == pytest.approx(ref, rel=1e-10, abs=1e-300)


@pytest.mark.parametrize("w,G,ax,ay,az", _rand_params(10, 2))
def test_signed_projected_area_identity(w, G, ax, ay, az):
    """sigma(-w) - sigma(w) = w . (0,0,G): Eq. spa with its right-hand side read
    as w . grad mu (equivalently Lambda(-w) = -1 - Lambda(w))."""
    a = oracle.projected_area_local(w, G, ax, ay, az)
    b = oracle.projected_area_local(-w, G, ax, ay, az)
    assert b - a == pytest.approx(G * w[2], abs=1e-13 * (1 + abs(a) + abs(b)))


@pytest.mark.parametrize("G,ax,ay,az", [(1.0, 0.5, 0.5, 0.5), (1.0, 0.3, 0.7, 1.2), (0.6, 1.0, 1.0, 1.0), (1.3, 2.0, 1.5, 0.4)])
def test_projected_area_is_vndf_normaliser(G, ax, ay, az):
    """int <-w, m> D(m) dm = sigma(w) (the equivalence shown numerically in the
    paper's figure on the generalized projected area; it is exact), with the
    paper's printed closed-form D."""
    RNG = np.random.default_rng(12)
    for _ in range(3):
        w = RNG.normal(size=3)
        w /= np.linalg.norm(w)
        pts, wts = H.sphere_points(-w, 96, 96, cos_range=(0.0, 1.0))  # hemisphere <-w,m> > 0
        D = H.ndf_paper_closed_form(pts, G, ax, ay, az)
        lhs = np.sum(wts * (pts @ -w) * D)
        assert oracle.projected_area_local(w, G, ax, ay, az) == pytest.approx(lhs, rel=1e-7)


@pytest.mark.parametrize("cos_t", [0.2, 0.5, 0.8, 0.97])
@pytest.mark.parametrize("alpha", [0.2, 0.6, 1.0])
def test_projected_area_reduces_to_beckmann_smith(cos_t, alpha):
    """alpha_z -> 0: sigma(w)/cos = Lambda_Beckmann(a = 1/(alpha tan)), the error
    shrinking like alpha_z^2 (text after Eq. generalized_lambda)."""
    w = np.array([math.sqrt(1 - cos_t ** 2), 0.0, cos_t])
    ref = H.beckmann_lambda(cos_t, alpha)
    errs = []
    for az in (1e-2, 1e-3):
        lam = oracle.projected_area_local(w, 1.0, alpha, alpha, az) / cos_t
        errs.append(abs(lam - ref) / max(abs(ref), 1e-300))
    a = cos_t / (alpha * math.sqrt(1 - cos_t ** 2))
    # the alpha_z correction to a^2 is O(alpha_z^2 a^2 / alpha^2)
    assert errs[1] < 1e-4 * max(1.0, a * a / alpha ** 2)
    assert errs[1] < errs[0] / 30 or errs[1] < 1e-12


# ------------------------------------------------------------- NDF D(m)
@pytest.mark.parametrize("w,G,ax,ay,az", _rand_params(20, 3))
def test_ndf_matches_scipy_quadrature_of_definition(w, G, ax, ay, az):
    """Eq. gdf_to_ndf by scipy's QUADPACK (a different quadrature) with Eq. gdf."""
    m = w

    def f(t):
        e = (t * m[0] / ax) ** 2 + (t * m[1] / ay) ** 2 + ((t * m[2] - G) / az) ** 2
        return t ** 3 * math.exp(-e) / (math.pi ** 1.5 * ax * ay * az)

    ref = quad(f, 0, np.inf, epsabs=0, epsrel=1e-13, limit=500)[0]
    assert oracle.ndf_local(m, G, ax, ay, az) == pytest.approx(ref, rel=1e-10, abs=1e-300)


@pytest.mark.parametrize("w,G,ax,ay,az", _rand_params(30, 4))
def test_ndf_matches_paper_closed_form(w, G, ax, ay, az):
    """Appendix A result (Eq. macro_ndf), where that printed form is well conditioned."""
    A = w[0] ** 2 / ax ** 2 + w[1] ** 2 / ay ** 2 + w[2] ** 2 / az ** 2
    q = G * w[2] / az ** 2 / math.sqrt(A)
    if q < -3:
        pytest.skip("printed closed form cancels here")
    ref = float(H.ndf_paper_closed_form(w, G, ax, ay, az))
    assert oracle.ndf_local(w, G, ax, ay, az) == pytest.approx(ref, rel=1e-11, abs=1e-300)


def test_appendix_terms_sum_to_the_integral():
    """Each of I1..I4 (Appendix A) against its numeric integral."""
    for (A, B) in [(1.3, 0.4), (0.7, -0.6), (4.0, 2.5), (2.0, 0.0)]:
        lo = -B / A
        nums = [quad(lambda u, k=k: u ** k * math.exp(-A * u * u), lo, np.inf, epsabs=0, epsrel=1e-13)[0] for k in (3, 2, 1, 0)]
        coef = [1.0, 3 * B / A, 3 * B * B / A ** 2, B ** 3 / A ** 3]
        for I, c, n in zip(H.appendix_terms(A, B), coef, nums):
            assert I == pytest.approx(c * n, rel=1e-10, abs=1e-14)


@pytest.mark.parametrize("ax,ay", [(0.3, 0.3), (0.2, 0.5), (0.8, 0.6)])
def test_ndf_reduces_to_beckmann(ax, ay):
    """alpha_z -> 0: D -> Beckmann NDF above the horizon and 0 below (text after Eq. macro_ndf)."""
    RNG = np.random.default_rng(13)
    for _ in range(6):
        m = RNG.normal(size=3)
        m[2] = abs(m[2]) + 0.4
        m /= np.linalg.norm(m)
        ref = H.beckmann_ndf(m, ax, ay)
        errs = [abs(oracle.ndf_local(m, 1.0, ax, ay, az) / ref - 1) for az in (1e-2, 1e-3)]
        assert errs[1] < 0.05 and (errs[1] < errs[0] / 30 or errs[1] < 1e-10)
        down = m * np.array([1, 1, -1])
        assert oracle.ndf_local(down, 1.0, ax, ay, 1e-3) < 1e-100


@pytest.mark.parametrize("G,ax,ay,az", [(1.0, 0.4, 0.4, 0.4), (1.0, 0.3, 0.8, 2.0), (0.5, 1.5, 1.5, 1.5)])
def test_oracle_ndf_signed_projected_area_on_sphere(G, ax, ay, az):
    """int (w.m) D(m) dm = w . (0,0,G) with the oracle's own quadrature D
    (Eq. spa, right-hand side read as w . grad mu)."""
    pts, wts = H.sphere_points(np.array([0.0, 0.0, 1.0]), 64, 96)
    D = np.array([oracle.ndf_local(m, G, ax, ay, az) for m in pts])
    for w in (np.array([0.0, 0.0, 1.0]), np.array([0.6, 0.0, 0.8])):
        assert np.sum(wts * (pts @ w) * D) == pytest.approx(G * w[2], rel=2e-6, abs=1e-9)
