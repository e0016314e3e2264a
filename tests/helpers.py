"""Test-side references that are independent of both the oracle and the CUDA path.

They are written from the paper's printed closed forms, textbook results and
scipy's special functions / quadrature, and serve as the pins the oracle is
checked against (the oracle itself computes D by quadrature of its definition
and sigma_t from its own C code).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sp
from numpy.polynomial.legendre import leggauss

from paper_2603_00280_gb300 import workloads as W


def ndf_paper_closed_form(m, G, ax, ay, az):
    """Appendix A final result (Eq. macro_ndf) with the mean gradient (0,0,G).

    The paper has G = 1; with mean (0,0,G) the same derivation gives B = G cos/az^2
    and C = G^2/az^2.  Well conditioned for B/sqrt(A) > -3 (cancellation below).
    """
    m = np.asarray(m, dtype=np.float64)
    m = m / np.linalg.norm(m, axis=-1, keepdims=True)
    A = m[..., 0] ** 2 / ax ** 2 + m[..., 1] ** 2 / ay ** 2 + m[..., 2] ** 2 / az ** 2
    B = G * m[..., 2] / az ** 2
    C = G * G / az ** 2
    q2 = B * B / A
    pre = np.exp(-C + q2) / (math.pi ** 1.5 * ax * ay * az)
    return pre * ((q2 + 1) * np.exp(-q2) / (2 * A * A)
                  + B * math.sqrt(math.pi) / (2 * A ** 2.5) * (q2 + 1.5) * sp.erfc(-B / np.sqrt(A)))


def appendix_terms(A, B):
    """I1..I4 of Appendix A as printed."""
    e = math.exp(-B * B / A)
    ec = sp.erfc(-B / math.sqrt(A))
    I1 = (B * B / (2 * A ** 3) + 1 / (2 * A * A)) * e
    I2 = -3 * B * B / (2 * A ** 3) * e + 3 * B * math.sqrt(math.pi) / (4 * A ** 2.5) * ec
    I3 = 3 * B * B / (2 * A ** 3) * e
    I4 = B ** 3 * math.sqrt(math.pi) / (2 * A ** 3.5) * ec
    return I1, I2, I3, I4


def beckmann_ndf(m, ax, ay):
    """Textbook anisotropic Beckmann NDF about +z (zero below the horizon)."""
    m = np.asarray(m, dtype=np.float64)
    m = m / np.linalg.norm(m)
    if m[2] <= 0:
        return 0.0
    return math.exp(-(m[0] ** 2 / ax ** 2 + m[1] ** 2 / ay ** 2) / m[2] ** 2) / (math.pi * ax * ay * m[2] ** 4)


def beckmann_lambda(cos_t, alpha):
    """Textbook Smith Lambda of the isotropic Beckmann NDF, a = 1/(alpha tan)."""
    a = cos_t / (alpha * math.sqrt(1 - cos_t * cos_t))
    return -math.erfc(a) / 2 + math.exp(-a * a) / (2 * a * math.sqrt(math.pi))


def frame(pole):
    z = np.asarray(pole, dtype=np.float64)
    z = z / np.linalg.norm(z)
    a = np.array([1.0, 0, 0]) if abs(z[0]) < 0.6 else np.array([0, 1.0, 0])
    x = a - np.dot(a, z) * z
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return x, y, z


def sphere_points(pole, n_theta=64, n_phi=128, cos_range=(-1.0, 1.0)):
    """Product rule on the sphere around ``pole``: Gauss-Legendre in cos(theta)
    over ``cos_range``, trapezoid (spectral for periodic integrands) in phi.
    Returns (directions (N,3), weights (N,))."""
    x, y, z = frame(pole)
    c, w = leggauss(n_theta)
    lo, hi = cos_range
    c = 0.5 * (hi - lo) * c + 0.5 * (hi + lo)
    w = 0.5 * (hi - lo) * w
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    cc, pp = np.meshgrid(c, phi, indexing="ij")
    ww = np.repeat(w[:, None], n_phi, axis=1) * (2 * math.pi / n_phi)
    s = np.sqrt(np.maximum(0.0, 1 - cc * cc))
    d = (s * np.cos(pp))[..., None] * x + (s * np.sin(pp))[..., None] * y + cc[..., None] * z
    return d.reshape(-1, 3), ww.reshape(-1)


def projected_area_by_quadrature(w, G, ax, ay, az):
    """E[max(0, -w.g)] for g ~ N((0,0,G), diag(alpha^2/2)) by 1-D quadrature of
    the Gaussian k = -w.g (the definition behind Eq. generalized_sigma_t)."""
    from scipy.integrate import quad
    w = np.asarray(w, dtype=np.float64)
    mean = -G * w[2]
    sd = math.sqrt(0.5 * (ax ** 2 * w[0] ** 2 + ay ** 2 * w[1] ** 2 + az ** 2 * w[2] ** 2))
    f = lambda k: k * math.exp(-0.5 * ((k - mean) / sd) ** 2) / (sd * math.sqrt(2 * math.pi))
    lo = max(0.0, mean - 40 * sd)
    return quad(f, lo, mean + 40 * sd, epsabs=0, epsrel=1e-13, limit=400, points=[max(lo, mean)] if mean > lo else None)[0]


# ------------------------------------------------------------------ slab scenes with exact grids

SLAB_SIGMA = 0.0625          # sigma^2 = 2^-8 exactly representable
SLAB_L = 1.0 / 32.0
SLAB_BMIN = (-0.5, -0.5, -0.125)
SLAB_BMAX = (0.5, 0.5, 0.125)


def dyadic_slab(albedo=0.75, light=None, mean="plane", nodes=(17, 17, 9), sigma=SLAB_SIGMA, l=SLAB_L):
    """Slab whose grid values are exact in float32: node spacing 1/16 x 1/16 x 1/32,
    mean = z (or a constant 0.0625), variance a power of two."""
    p = W.node_coords(SLAB_BMIN, SLAB_BMAX, nodes)
    mu = p[..., 2] if mean == "plane" else np.full(p.shape[:3], float(mean))
    obj = W.make_object(mu, sigma * sigma, albedo, SLAB_BMIN, SLAB_BMAX, l)
    return {"objects": [obj], "light": light or W.directional_light((0.0, 0.0, 1.0), 1.0)}


def slab_projected_area(d, sigma=SLAB_SIGMA, l=SLAB_L, slope=1.0):
    """sigma(d) for the plane mean mu = slope * z (grad = (0,0,slope)); textbook
    E[max(0,X)], X ~ N(m, s^2) = m Phi(m/s) + s phi(m/s) with m = -slope d_z, s = sigma/l."""
    s = sigma / l
    m = -slope * d[2]
    return m * sp.ndtr(m / s) + s * math.exp(-0.5 * (m / s) ** 2) / math.sqrt(2 * math.pi)


def slab_optical_depth(z0, z1, d, sigma=SLAB_SIGMA, l=SLAB_L, slope=1.0):
    """Optical depth between heights z0 and z1 along d for the plane mean mu = slope z:
    int lambda(u) du = ln Phi(u) with u = slope z/sigma, so
    tau = sigma(d)/(slope d_z) (lnPhi(slope z1/sigma) - lnPhi(slope z0/sigma))."""
    return slab_projected_area(d, sigma, l, slope) / (slope * d[2]) * (
        sp.log_ndtr(slope * z1 / sigma) - sp.log_ndtr(slope * z0 / sigma))


def slab_single_scatter(d, wl, albedo, sigma=SLAB_SIGMA, l=SLAB_L, irradiance=1.0, ztop=0.125, zbot=-0.125, shift=0.0,
                        slope=1.0):
    """Exact single-scattered radiance for a ray entering the slab top along d
    (d_z < 0) and leaving through the bottom, lit by a directional light from
    wl (wl_z > 0, leaving through the top).  p is constant along the ray, so
    L = int Tr_cam sigma_t p Tr_light E dt is a 1-D integral of closed forms.
    `shift` moves the mean to mu = slope (z + shift) (the box stays put); `slope`
    scales the plane mean's gradient to (0, 0, slope)."""
    from scipy.integrate import quad
    alpha = math.sqrt(2) * sigma / l
    m = np.asarray(wl) - np.asarray(d)
    m /= np.linalg.norm(m)
    sd = slab_projected_area(d, sigma, l, slope)
    D = ndf_paper_closed_form(np.array([math.sqrt(max(0, 1 - m[2] ** 2)), 0, m[2]]), slope, alpha, alpha, alpha)
    p = albedo * D / (4 * sd)

    def f(z):
        u = slope * (z + shift) / sigma
        rho = math.exp(-0.5 * u * u - 0.5 * math.log(2 * math.pi) - sp.log_ndtr(u)) / sigma
        tau_c = slab_optical_depth(ztop + shift, z + shift, d, sigma, l, slope)
        tau_l = slab_optical_depth(z + shift, ztop + shift, wl, sigma, l, slope)
        return math.exp(-tau_c - tau_l) * rho * sd * p * irradiance / abs(d[2])

    return quad(f, zbot, ztop, epsabs=0, epsrel=1e-12, limit=400)[0]


def slab_single_scatter_objects(d, wl, objects, irradiance=1.0, ztop=0.125, zbot=-0.125):
    """Exact single scattering (as slab_single_scatter) in a slab holding several
    co-located plane-mean objects, each a tuple (albedo, sigma, l): extinctions add
    along both rays, and the scattered radiance at height z is the sum over objects
    of sigma_t,k(z) p_k (each object scatters with its own phase function and albedo)."""
    from scipy.integrate import quad
    m = np.asarray(wl) - np.asarray(d)
    m /= np.linalg.norm(m)
    mloc = np.array([math.sqrt(max(0, 1 - m[2] ** 2)), 0, m[2]])
    terms = []
    for F, sig, l in objects:
        alpha = math.sqrt(2) * sig / l
        sd = slab_projected_area(d, sig, l)
        D = ndf_paper_closed_form(mloc, 1.0, alpha, alpha, alpha)
        terms.append((F * D / (4 * sd), sd, sig, l))

    def f(z):
        tau = 0.0
        scat = 0.0
        for p, sd, sig, l in terms:
            tau += slab_optical_depth(ztop, z, d, sig, l) + slab_optical_depth(z, ztop, wl, sig, l)
            u = z / sig
            rho = math.exp(-0.5 * u * u - 0.5 * math.log(2 * math.pi) - sp.log_ndtr(u)) / sig
            scat += rho * sd * p
        return math.exp(-tau) * scat * irradiance / abs(d[2])

    return quad(f, zbot, ztop, epsabs=0, epsrel=1e-12, limit=400)[0]


def zscores(mean_a, se_a, mean_b, se_b=0.0):
    return (np.asarray(mean_a) - np.asarray(mean_b)) / np.sqrt(np.asarray(se_a) ** 2 + np.asarray(se_b) ** 2)


def tiny_brute_force_scene():
    """A 3x3x3-node heterogeneous GPSS (noisy sphere mean, random variance) lit by a
    directional light, and a 4x4 orthographic camera: the brute-force input on which the
    oracle's regular tracking is checked against a naive delta tracker, and the GPU
    against the oracle."""
    rng = np.random.default_rng(7)
    lo, hi = np.array([-0.25, -0.25, -0.25]), np.array([0.25, 0.25, 0.25])
    p = W.node_coords(lo, hi, (3, 3, 3))
    mean = (W.sdf_sphere(p, (0.0, 0.0, 0.0), 0.15) + rng.uniform(-0.03, 0.03, p.shape[:3])).astype(np.float32)
    var = rng.uniform(0.02 ** 2, 0.05 ** 2, p.shape[:3]).astype(np.float32)
    sc = {"objects": [W.make_object(mean, var, 0.8, lo, hi, 0.05)],
          "light": W.directional_light((0.3, -0.4, 1.0), 1.0)}
    cam = {"type": "ortho", "eye": (0.0, -1.0, 0.35), "look_at": (0.0, 0.0, 0.0), "up": (0.0, 0.0, 1.0),
           "fov_y_deg": 40.0, "ortho_w": 0.45, "ortho_h": 0.45, "width": 4, "height": 4}
    return sc, cam, lo, hi
