"""Writes moment_fit.inc: Chebyshev coefficients of ln M3(q) and ln M4(q) on
q in [-3, 0], where M_k(q) = int_0^inf s^k exp(-s^2 + 2 q s) ds are the moments
behind the closed-form NDF of the GPSS (Appendix A of the paper, rearranged).

In that range the three-term recurrence M_{k+1} = q M_k + (k/2) M_{k-1} cancels
badly in FP32 (it amplifies the error of M0 = sqrt(pi)/2 erfcx(-q) up to ~75x at
q = -1.5), and the continued fraction of M_k/M_{k-1} converges slowly, so the
device evaluates a fitted polynomial there instead.  The fit is computed here in
FP64 (recurrence seeded with scipy's erfcx, whose cancellation costs < 1e-13 in
double) at 400 Chebyshev points; degree 10 gives a fit error below 2e-9.

    python gen_moment_fit.py     # rewrites moment_fit.inc next to this script
"""
import math
import os

import numpy as np
import scipy.special as sp
from numpy.polynomial import chebyshev as ch

LO, HI, DEG = -3.0, 0.0, 10


def moment(k, q):
    m = [0.5 * math.sqrt(math.pi) * sp.erfcx(-q)]
    m.append(q * m[0] + 0.5)
    for j in range(1, k):
        m.append(q * m[j] + 0.5 * j * m[j - 1])
    return m[k]


def fit(k):
    xs = np.cos(np.pi * (np.arange(400) + 0.5) / 400)
    qs = LO + (xs + 1) * (HI - LO) / 2
    c = ch.chebfit(xs, np.log([moment(k, q) for q in qs]), DEG)
    qt = np.linspace(LO, HI, 4001)
    err = np.max(np.abs(np.exp(ch.chebval(2 * (qt - LO) / (HI - LO) - 1, c)) / np.array([moment(k, q) for q in qt]) - 1))
    return c, err


def main():
    lines = ["// Generated by gen_moment_fit.py -- do not edit.",
             "// Chebyshev coefficients (first kind, x = 2 (q - %g) / %g - 1) of ln M3(q) and ln M4(q)" % (LO, HI - LO),
             "// on q in [%g, %g]; M_k(q) = int_0^inf s^k exp(-s^2 + 2 q s) ds." % (LO, HI)]
    for k in (3, 4):
        c, err = fit(k)
        lines.append("// max relative fit error of M%d: %.2e" % (k, err))
        lines.append("constexpr int kMomentFitDeg = %d;" % DEG if k == 3 else "")
        body = ", ".join("%.9ef" % v for v in c)
        lines.append("__device__ __constant__ float c_lnM%d_cheb[%d] = {%s};" % (k, DEG + 1, body))
    lines.append("constexpr float kMomentFitLo = %.1ff, kMomentFitHi = %.1ff;" % (LO, HI))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "moment_fit.inc")
    open(out, "w").write("\n".join(l for l in lines if l) + "\n")
    print(out)


if __name__ == "__main__":
    main()
