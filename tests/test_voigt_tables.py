"""Host-side check of the device Voigt approximation's tables (no GPU).

The CUDA path evaluates H(a, x) from two generated tables (csrc/voigt_coeffs.h): the
degree-11 fits of K(x) = 2 x F(x) - 1 on six unit intervals (|x| < 6) and the degree-4
wing polynomial g(t), t = 1/(x^2 + a^2) (|x| >= 6).  Evaluated here in float64 with the
same formulas, they must reproduce H = Re w(x + i a) (scipy's Faddeeva function) to a
few 1e-7, which leaves the FP32 kernels inside their 1e-5 budget."""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2507_11603_gb300", "csrc", "voigt_coeffs.h")


def tables():
    txt = open(HDR).read()
    rows = re.findall(r"\{([^{}]*)\},", txt)
    K = np.array([[float(v.rstrip("f")) for v in r.split(",")] for r in rows])
    W = np.array([float(v) for v in re.findall(r"THOR_WING_C\d (\S+)f", txt)])
    return K, W


def h_tables(a, x):
    K, W = tables()
    ax = np.abs(x)
    x2 = ax * ax
    i = np.minimum(ax.astype(int), K.shape[0] - 1)
    u = ax - (i + 0.5)
    k = np.zeros_like(ax)
    for j in range(K.shape[1] - 1, -1, -1):
        k = k * u + K[i, j]
    core = (np.exp(-x2) * (1 + a * a * (1 - 2 * x2)) + 2 * a / np.sqrt(np.pi) * k
            + a ** 3 / (3 * np.sqrt(np.pi)) * ((6 - 4 * x2) * k + 2))
    t = 1.0 / (x2 + a * a)
    g = np.zeros_like(t)
    for c in W[::-1]:
        g = g * t + c
    wing = a / np.sqrt(np.pi) * t * g
    return np.where(ax >= 6.0, wing, core)


@pytest.mark.parametrize("a", [5e-5, 4.7e-4, 2e-3, 1e-2])
def test_device_voigt_tables_against_faddeeva(a):
    from scipy.special import wofz
    x = np.concatenate([np.linspace(0.0, 12.0, 24001), np.geomspace(12.0, 300.0, 4001)])
    ref = wofz(x + 1j * a).real
    rel = np.abs(h_tables(a, x) - ref) / ref
    assert rel.max() < 1e-6, (a, rel.max(), x[np.argmax(rel)])


def test_wing_polynomial_matches_series_limit():
    # g(t) -> 1 + 3t/2 + 15t^2/4 + ... as t -> 0 (the asymptotic series of w)
    _, W = tables()
    assert abs(W[0] - 1.0) < 1e-6 and abs(W[1] - 1.5) < 1e-3


def test_core_polynomial_against_faddeeva():
    """The single core polynomial (|x| <= 2, no table lookup) of the photon loops' fast core
    path: K(x) = sum_j p_j (x^2/4)^j in float64 with the same series in a reproduces
    H = Re w(x + i a) to 3e-6 relative for a in [5e-5, 1e-2]."""
    from scipy.special import wofz
    txt = open(HDR).read()
    p = np.array([float(v) for v in re.findall(r"THOR_VCORE_P\d (\S+)f", txt)])
    assert p.size == 9
    x = np.linspace(-2.0, 2.0, 8001)
    s = x * x / 4.0
    k = np.zeros_like(s)
    for c in p[::-1]:
        k = k * s + c
    for a in (5e-5, 4.7e-4, 2e-3, 1e-2):
        x2 = x * x
        h = (np.exp(-x2) * (1 + a * a * (1 - 2 * x2)) + 2 * a / np.sqrt(np.pi) * k
             + a ** 3 / (3 * np.sqrt(np.pi)) * ((6 - 4 * x2) * k + 2))
        assert np.max(np.abs(h / wofz(x + 1j * a).real - 1)) < 3e-6, a
