"""Generate the coefficient table of the device Voigt approximation (voigt_coeffs.h).

The device evaluates H(a,x) for |x| < 6 as
    H = exp(-x^2) (1 + a^2 (1 - 2x^2)) + (2a/sqrt(pi)) K(x) + (a^3/(3 sqrt(pi))) ((6 - 4x^2) K(x) + 2)
with K(x) = 2 x F(x) - 1 and F Dawson's integral (the Taylor series of w(x + i a) in a,
truncated after a^3).  K is fitted here, per unit interval [i, i+1), i = 0..5, by a
degree-11 polynomial in u = x - (i + 1/2) (least squares on Chebyshev nodes, float64,
F from scipy.special.dawsn).

For |x| <= 2 the photon loops' fast core path uses one polynomial instead of the table:
K(x) = sum_j p_j s^j with s = x^2 / 4, j = 0..8 (K is even; least squares on Chebyshev
nodes in s; max error 4.5e-6 in K, 2e-6 relative in H for a <= 1e-2), evaluated without
a table lookup.

For |x| >= 6 the device uses H = (a/sqrt(pi)) t g(t), t = 1/(x^2 + a^2), where
g(t) = 2 x^2 K(x) at x = t^(-1/2) (the a-linear term; the a^3 term is below 1.5 a^2/x^2
relative) is fitted on t in (0, 1/36] by a degree-4 polynomial (relative least squares on
Chebyshev nodes; max relative error 4e-8, better than eight terms of the asymptotic
series at x = 6).  Deterministic: re-running reproduces voigt_coeffs.h.
"""
import os

import numpy as np
from scipy.special import dawsn

DEG = 11
NINT = 6


def K(x):
    return 2.0 * x * dawsn(x) - 1.0


def fit():
    rows = []
    for i in range(NINT):
        c = i + 0.5
        t = np.cos(np.pi * (np.arange(400) + 0.5) / 400)
        x = c + 0.5 * t
        u = x - c
        V = np.vander(u, DEG + 1, increasing=True)
        # weight: relative in the tail where K ~ 1/(2x^2), absolute near the zero of K
        w = 1.0 / np.maximum(np.abs(K(x)), 1e-2)
        coef, *_ = np.linalg.lstsq(V * w[:, None], K(x) * w, rcond=None)
        rows.append(coef)
    return np.array(rows)


WING_DEG = 4


def fit_wing():
    n = 2000
    t = (1.0 / 36.0) * (0.5 + 0.5 * np.cos(np.pi * (np.arange(n) + 0.5) / n))
    x = 1.0 / np.sqrt(t)
    g = 2.0 * x * x * K(x)
    V = np.vander(t, WING_DEG + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(V / g[:, None], np.ones_like(g), rcond=None)
    return coef


CORE_DEG = 8
CORE_X = 2.0


def fit_core():
    n = 4000
    t = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    s = 0.5 + 0.5 * t
    x = CORE_X * np.sqrt(s)
    V = np.vander(s, CORE_DEG + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(V, K(x), rcond=None)
    return coef


def main():
    rows = fit()
    wing = fit_wing()
    core = fit_core()
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "voigt_coeffs.h"), "w") as f:
        f.write("// Generated by gen_voigt_coeffs.py -- do not edit.\n")
        f.write("// K(x) = 2 x F(x) - 1 on [i, i+1): sum_j c[i][j] (x - i - 1/2)^j, j = 0..11\n")
        f.write("#pragma once\n")
        f.write(f"#define THOR_VOIGT_NINT {NINT}\n#define THOR_VOIGT_NCOEF {DEG + 1}\n")
        f.write("static const float kVoigtK[THOR_VOIGT_NINT][THOR_VOIGT_NCOEF] = {\n")
        for r in rows:
            f.write("  {" + ", ".join(f"{v:.9e}f" for v in r) + "},\n")
        f.write("};\n")
        f.write("// |x| >= 6: H = (a/sqrt(pi)) t sum_j w_j t^j, t = 1/(x^2 + a^2), j = 0..4\n")
        for j, v in enumerate(wing):
            f.write(f"#define THOR_WING_C{j} {v:.9e}f\n")
        f.write(f"// |x| <= {CORE_X:g}: K(x) = sum_j p_j s^j, s = x^2 / {CORE_X * CORE_X:g}, j = 0..{CORE_DEG}\n")
        f.write(f"#define THOR_VCORE_X {CORE_X:.1f}f\n")
        for j, v in enumerate(core):
            f.write(f"#define THOR_VCORE_P{j} {v:.9e}f\n")


if __name__ == "__main__":
    main()
