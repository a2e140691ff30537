"""Closed forms and independent numerics that pin the oracle (test helpers only).

Nothing here shares code with the oracle or with the CUDA path: special functions
come from scipy / mpmath, integrals from scipy.integrate.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, special

SQRT_PI = np.sqrt(np.pi)


def voigt_scipy(a, x):
    """H(a,x) = Re w(x + i a) via scipy's Faddeeva function (MIT package)."""
    return special.wofz(np.asarray(x) + 1j * np.asarray(a)).real


def neufeld_sphere_shape(x, a_tau0):
    """Emergent spectrum of a static uniform sphere with a central source at line
    centre, a tau0 >> 1 (Dijkstra, Haiman & Spaans 2006):
    J(x) ~ x^2 / (1 + cosh(sqrt(2 pi^3 / 27) |x|^3 / (a tau0)))."""
    x = np.asarray(x, dtype=float)
    y = np.minimum(np.sqrt(2.0 * np.pi ** 3 / 27.0) * np.abs(x) ** 3 / a_tau0, 700.0)
    return x * x / (1.0 + np.cosh(y))


def neufeld_slab_shape(x, a_tau0):
    """Emergent spectrum of a static slab, central source, a tau0 >> 1 (Neufeld 1990):
    J(x) ~ x^2 / cosh(sqrt(pi^3 / 54) |x|^3 / (a tau0))."""
    x = np.asarray(x, dtype=float)
    y = np.minimum(np.sqrt(np.pi ** 3 / 54.0) * np.abs(x) ** 3 / a_tau0, 700.0)
    return x * x / np.cosh(y)


def binned_expectation(shape, edges, n_total, **kw):
    """Expected counts per bin for a density proportional to shape(x), normalised to n_total."""
    lo, hi = edges[0], edges[-1]
    norm = integrate.quad(lambda t: shape(t, **kw), lo, hi, limit=400)[0]
    out = np.array([integrate.quad(lambda t: shape(t, **kw), edges[i], edges[i + 1])[0]
                    for i in range(len(edges) - 1)])
    return n_total * out / norm


def laursen_fesc(a_tau0, tau_a, zeta=0.525):
    """Escape fraction from a dusty slab, central source at line centre
    (Neufeld 1990 form with the fitted constant of Laursen, Razoumov & Sommer-Larsen 2009):
    f_esc = 1 / cosh( sqrt(3) / (zeta pi^(5/12)) * sqrt((a tau0)^(1/3) tau_a) )."""
    return 1.0 / np.cosh(np.sqrt(3.0) / (zeta * np.pi ** (5.0 / 12.0)) * np.sqrt(a_tau0 ** (1.0 / 3.0) * tau_a))


def hummer_RIA_conditional(x_out, x_in):
    """Frequency redistribution after one scattering with isotropic phase function,
    pure Doppler broadening (a -> 0), no recoil (Hummer 1962, R_I-A):
    p(x_out | x_in) = (sqrt(pi)/2) exp(x_in^2) erfc(max(|x_in|, |x_out|))."""
    return 0.5 * SQRT_PI * np.exp(x_in ** 2) * special.erfc(np.maximum(np.abs(x_in), np.abs(x_out)))


def dipole_redistribution(x_out, x_in):
    """Same limit as above with the dipole phase function P(mu) = 3/8 (1 + mu^2):
    the atom moves with u_par = x_in along k_in and N(0, 1/2) perpendicular components,
    so x_out | mu ~ N(x_in mu, (1 - mu^2)/2); integrate over mu numerically."""
    x_out = np.atleast_1d(np.asarray(x_out, dtype=float))
    mu, w = np.polynomial.legendre.leggauss(400)
    var = np.maximum((1.0 - mu ** 2) / 2.0, 1e-300)
    P = 0.375 * (1.0 + mu ** 2)
    dens = np.exp(-(x_out[:, None] - x_in * mu[None, :]) ** 2 / (2 * var)) / np.sqrt(2 * np.pi * var)
    return (dens * (P * w)[None, :]).sum(axis=1)


def upar_density(u, x, a):
    """Unnormalised Eq. (6): exp(-u^2) / ((x - u)^2 + a^2)."""
    return np.exp(-u * u) / ((x - u) ** 2 + a * a)


def upar_cdf_table(x, a, lo=-8.0, hi=None):
    """Numerically integrated CDF of Eq. (6) on a grid refined around the resonance u = x."""
    hi = max(8.0, abs(x) + 8.0) if hi is None else hi
    pts = sorted({lo, hi, x - 50 * a, x - 5 * a, x, x + 5 * a, x + 50 * a, 0.0})
    pts = [p for p in pts if lo <= p <= hi]
    grid = [np.linspace(pts[i], pts[i + 1], 4001) for i in range(len(pts) - 1)]
    u = np.unique(np.concatenate(grid))
    f = upar_density(u, x, a)
    # cumulative integral piecewise with Simpson-quality refinement through quad per node gap
    c = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(u))])
    return u, c / c[-1]


def upar_mean(x, a):
    """E[u_par] by adaptive quadrature of Eq. (6)."""
    pts = [x - 10 * a, x, x + 10 * a]
    f = lambda u: upar_density(u, x, a)
    g = lambda u: u * upar_density(u, x, a)
    lo, hi = -12.0, abs(x) + 12.0
    num = integrate.quad(g, lo, hi, points=pts, limit=500, epsabs=0, epsrel=1e-10)[0]
    den = integrate.quad(f, lo, hi, points=pts, limit=500, epsabs=0, epsrel=1e-10)[0]
    return num / den


# ----------------------------------------------------------------------- dust scattering
def hg_density(mu, g):
    """Henyey-Greenstein phase function per unit mu on [-1, 1] (Eq. 9)."""
    return 0.5 * (1.0 - g * g) / (1.0 + g * g - 2.0 * g * mu) ** 1.5


def dust_sphere_first_orders(kappa, g):
    """Uniform dust sphere of radius 1 with extinction kappa per unit length (no gas
    opacity) and a central point source.  Returns (P0, I1): P0 = exp(-kappa), the chance of
    leaving without an interaction, and I1, the chance of leaving right after exactly one
    interaction if that interaction always scatters (Eq. 8 with albedo 1):
        I1 = int_0^1 kappa e^{-kappa r} int_{-1}^{1} p_HG(mu) e^{-kappa L(r, mu)} dmu dr,
    L(r, mu) = -r mu + sqrt(1 - r^2 (1 - mu^2)) the distance to the surface from radius r
    along a direction at cosine mu to the (radial) incoming direction."""
    def inner(mu, r):
        L = -r * mu + np.sqrt(max(0.0, 1.0 - r * r * (1.0 - mu * mu)))
        return kappa * np.exp(-kappa * r) * hg_density(mu, g) * np.exp(-kappa * L)
    I1 = integrate.dblquad(inner, 0.0, 1.0, -1.0, 1.0, epsabs=1e-12, epsrel=1e-10)[0]
    return float(np.exp(-kappa)), float(I1)


def _box_exit(p, k, side):
    """Distance from points p inside [0, side]^3 along unit directions k to the box surface."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(k > 0, (side - p) / k, np.where(k < 0, -p / k, np.inf))
    return t.min(axis=1)


def _iso_dirs(u1, u2):
    mu = 2.0 * u1 - 1.0
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    ph = 2.0 * np.pi * u2
    return np.stack([st * np.cos(ph), st * np.sin(ph), mu], axis=1)


def dust_cube_first_orders(kappa, side, g, m=20, seed=0):
    """Uniform dust cube [0, side]^3 with extinction kappa per unit length, sources uniform
    in the volume and isotropic.  Returns (P0, I1) as dust_sphere_first_orders does, by
    scrambled Sobol quadrature over (position, direction) for P0 (5 dimensions) and
    (position, direction, flight to the first interaction, scattering mu and phi) for I1
    (8 dimensions, 2^m points).  The flight length is drawn from the exponential truncated at
    the exit distance (weight 1 - e^{-kappa L0}), and mu uniformly on [-1, 1] with the weight
    2 p_HG(mu), so the phase function enters only through its density."""
    from scipy.stats import qmc
    u = qmc.Sobol(d=5, scramble=True, seed=seed).random_base2(m)
    p = side * u[:, :3]
    k = _iso_dirs(u[:, 3], u[:, 4])
    P0 = float(np.mean(np.exp(-kappa * _box_exit(p, k, side))))
    u = qmc.Sobol(d=8, scramble=True, seed=seed + 1).random_base2(m)
    p = side * u[:, :3]
    k = _iso_dirs(u[:, 3], u[:, 4])
    L0 = _box_exit(p, k, side)
    w = -np.expm1(-kappa * L0)
    r = -np.log1p(-u[:, 5] * w) / kappa
    p1 = p + r[:, None] * k
    mu = 2.0 * u[:, 6] - 1.0
    ph = 2.0 * np.pi * u[:, 7]
    # orthonormal pair perpendicular to k (cross products with the least aligned axis)
    ref = np.zeros_like(k)
    ref[np.arange(len(k)), np.argmin(np.abs(k), axis=1)] = 1.0
    e1 = np.cross(k, ref)
    e1 /= np.linalg.norm(e1, axis=1)[:, None]
    e2 = np.cross(k, e1)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    k1 = mu[:, None] * k + st[:, None] * (np.cos(ph)[:, None] * e1 + np.sin(ph)[:, None] * e2)
    I1 = float(np.mean(w * 2.0 * hg_density(mu, g) * np.exp(-kappa * _box_exit(p1, k1, side))))
    return P0, I1


def dust_event_order_probabilities(P0, I1, albedo):
    """Chances of (dust scatterings, fate) for a photon that interacts only with dust of
    albedo A (Eq. 8), from P0 and I1: each interaction scatters with probability A.
    Keys: (0, 'esc'), (0, 'abs'), (1, 'esc'), (1, 'abs'), ('2+', None)."""
    A = albedo
    return {(0, "esc"): P0, (0, "abs"): (1.0 - A) * (1.0 - P0), (1, "esc"): A * I1,
            (1, "abs"): A * (1.0 - A) * (1.0 - P0 - I1), ("2+", None): A * A * (1.0 - P0 - I1)}
