"""Algorithmic FP32 work of the hot path, tallied from the written formulas.

This is the numerator of the benchmark's FP32-issue roofline: what the method has
to compute per extinction evaluation and per real path vertex, counted from the
paper's formulas as this library evaluates them (not from the compiled code, and
not counting what an implementation wastes: loop control, index arithmetic,
traversal of empty space, random-number generation, divergence).

Counting rules (one "op" = one FP32 lane operation, the unit of the roofline's
peak of 128 lanes x SMs x clock):
  - add, sub, mul, fma, min/max, compare: 1 (an FMA counts once, as in the peak);
  - div, rcp, sqrt, rsqrt, exp, log, sin/cos: 1 (one special-function-unit issue);
  - erfc / erfcx / erf of FP32 accuracy: 12 (a degree-8 rational or polynomial
    kernel and its exponential: 10 FMA, 1 rcp, 1 exp);
  - lerp(a, b, t) = fma(t, b - a, a): 2.
Each formula below lists its steps and their counts; ``tally()`` sums them and
``python -m paper_2603_00280_gb300.opcounts`` writes opcounts.json beside this
file, which bench.py reads.

Passages: field fetch (Sec. 4: the normal is the normalised gradient of the mean
SDF; node-centred trilinear grids, reading Q12); extinction (Eq. generalized_sigma_t,
Eq. generalized_lambda, Eq. macro_sigma_t); delta and ratio tracking (Sec. 5); NDF
(Eq. gdf_to_ndf, Eq. gdf, Eq. macro_ndf, Appendix A); phase function and sampling
mixture (Eq. phase, Eq. microfacet_vndf, end of Sec. 4.2).
"""
from __future__ import annotations

import json
import os

ERFC = 12
LERP = 2

# (step, ops) per formula
FORMULAS = {
    # ---- per tentative collision (real, null or shadow): A1 + A2 + the tracking step
    "field_fetch": [
        ("cell coordinates f = (x - bmin) * inv_h, 3 axes", 6),
        ("cell index floor, 3 axes", 3),
        ("trilinear weights w = f - floor(f), 3 axes", 3),
        ("mean: 7 lerps over the 8 corners", 7 * LERP),
        ("grad mu x: 4 corner differences, 3 lerps, scale by inv_h", 4 + 3 * LERP + 1),
        ("grad mu y: 2 differences of the x-interpolants, 1 lerp, scale", 2 + LERP + 1),
        ("grad mu z: 1 difference, scale", 2),
        ("variance: 7 lerps", 7 * LERP),
    ],
    "extinction": [
        ("sigma = sqrt(var)", 1),
        ("u = mu / sigma", 1),
        ("lambda(u) = sqrt(2/pi) / erfcx(-u/sqrt2): scale, erfcx, div", 1 + ERFC + 1),
        ("rho = lambda / sigma", 1),
        ("alpha = sigma * sqrt2 / l", 1),
        ("a = (d . grad mu) / alpha: dot, div", 3 + 1),
        ("exp(-a^2) with the error-free square: mul, fma, exp, 2 corrections", 5),
        ("erfc(a) from erfcx(|a|) e^{-a^2}: erfcx, mul, select", ERFC + 2),
        ("psi(a) = e^{-a^2}/(2 sqrt pi) - (a/2) erfc(a)", 3),
        ("sigma(d) = alpha psi(a)", 1),
        ("sigma_t = rho sigma(d)", 1),
    ],
    "tracking_step": [
        ("tentative distance t += -ln(u) / majorant: log, div, add", 3),
        ("position x = o + t d", 3),
        ("real / null decision u' * majorant < sigma_t, or ratio T *= 1 - sigma_t/majorant", 3),
    ],
    # ---- per real vertex: A6 phase sampling + evaluation, A5 NEE evaluation + MIS
    "vertex_setup": [
        ("object field at the vertex (shared by sample and NEE): fetch", None),  # = field_fetch, added in tally()
        ("sigma(d) of the arriving direction (shared)", 1 + 1 + 4 + 5 + ERFC + 2 + 3 + 1),
        ("albedo: 7 lerps per channel, 3 channels", 3 * 7 * LERP),
        ("Beckmann proposal frame z = sign(-d.n) n and roughness alpha/|g| (norm, rsqrt, 4)", 3 + 1 + 4 + 2),
        ("Beckmann visible normaliser (1 + Lambda(w_i)) cos: cos, sin, a, erf, exp, combine", 2 + 2 + 2 + ERFC + 2 + 5),
    ],
    "ndf": [
        ("q = (m . grad mu) / alpha", 4),
        ("|grad mu x m|^2: cross, dot", 6 + 3),
        ("E = exp(-b^2/alpha^2) (or exp(-|g|^2/alpha^2))", 3),
        ("M0 = sqrt(pi)/2 erfcx term, M1, M2, M3 by the forward recurrence", ERFC + 2 + 3 * 2),
        ("D = alpha E M3 / pi^(3/2)", 3),
    ],
    "mixture_pdf": [
        ("Beckmann NDF about z: cos, cos^2, tan^2/alpha^2, exp, normalise", 2 + 1 + 3 + 1 + 3),
        ("visible density <w_i, m> D_B / normaliser", 3 + 2),
        ("mixture R pdf_B + (1 - R)/(2 pi)", 2),
        ("pdf over d' = pdf_m / (4 |d . m|)", 3 + 2),
    ],
    "phase_sample": [
        ("three uniforms to floats", 3),
        ("stretch w_i by the roughness, normalise, polar angles", 6 + 3 + 4),
        ("slope x: bracketed Newton on C(x) = cot (1 + erf x)/2 + e^{-x^2}/(2 sqrt pi), 6 steps",
         6 * (ERFC + 2 + 6)),
        ("slope y = erfinv(2u - 1)", ERFC + 2),
        ("rotate, unstretch, slope -> normal, to world", 4 + 2 + 4 + 9),
        ("uniform-hemisphere alternative: cos, sin, to world (R-weighted: half the draws)", (2 + 2 + 9) // 2),
        ("reflect d' = d - 2 (d.m) m", 6),
        ("weight F D |d.m| / (sigma(d) pdf_m) and throughput update, 3 channels", 4 + 6),
    ],
    "nee": [
        ("light direction uniform on the sphere: z, r = sqrt(1 - z^2), sincos", 2 + 3 + 2 + 2),
        ("half vector m = normalize(w_L - d)", 3 + 5),
        ("sky radiance lerp, 3 channels", 3 * LERP),
        ("p = F D/(4 sigma(d)) and MIS power heuristic", 3 + 5),
        ("contribution beta F p Le w / pdf_L, 3 channels; added to L after the shadow ray", 9 + 3),
    ],
}


def tally():
    """Per-function sums and the two totals the roofline uses."""
    sums = {}
    for name, steps in FORMULAS.items():
        sums[name] = sum(c for _, c in steps if c is not None)
    sums["vertex_setup"] += sums["field_fetch"]
    per_eval = sums["field_fetch"] + sums["extinction"] + sums["tracking_step"]
    # a vertex: its shared set-up, one NDF + mixture pdf for the sampled direction, one
    # NDF + mixture pdf (MIS) for the NEE direction, the sample itself and the NEE terms
    per_vertex = (sums["vertex_setup"] + 2 * (sums["ndf"] + sums["mixture_pdf"]) + sums["phase_sample"]
                  + sums["nee"])
    return {"per_function": sums, "ops_per_extinction_evaluation": per_eval, "ops_per_vertex_shading": per_vertex,
            "bytes_per_extinction_evaluation": 64,
            "rules": "FP32 lane operations; FMA = 1; div/sqrt/exp/log/sincos = 1; erfc/erfcx/erf = %d; lerp = %d"
                     % (ERFC, LERP),
            "formulas": {k: [[s, c] for s, c in v] for k, v in FORMULAS.items()}}


PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "opcounts.json")


def load():
    """The committed tally (opcounts.json)."""
    with open(PATH) as fh:
        return json.load(fh)


if __name__ == "__main__":
    t = tally()
    with open(PATH, "w") as fh:
        json.dump(t, fh, indent=1)
    print("per extinction evaluation: %d ops; per vertex: %d ops -> %s"
          % (t["ops_per_extinction_evaluation"], t["ops_per_vertex_shading"], PATH))
