"""Pins of the oracle's dust scattering in transport (albedo > 0; Sec. 2.3.2, Eq. 8-9).

A photon in a medium where only dust interacts scatters at each interaction with
probability A (the albedo, Eq. 8) into a Henyey-Greenstein direction (Eq. 9), or is
absorbed.  Sorting photons by (number of dust scatterings, fate) gives chances that
follow from two numbers of the geometry alone: P0, the chance to leave without an
interaction, and I1, the chance to leave right after one interaction that scatters
(`analytic.dust_event_order_probabilities`).  Both are computed here without the oracle:
by scipy quadrature for a sphere with a central source, by Sobol quadrature for a cube
with sources spread through it.

Each test also checks that the counts reject the same model with the albedo test turned
round (A -> 1 - A) and with the HG angle mirrored (g -> -g), so a planted mistake of either
kind in the oracle fails it.
"""
import numpy as np
import pytest

from tests import analytic as A

CATS = [(0, "esc"), (0, "abs"), (1, "esc"), (1, "abs"), ("2+", None)]


def _observed(ndust, status):
    nd = np.asarray(ndust).astype(np.int64)
    st = np.asarray(status)
    return {(0, "esc"): np.sum((nd == 0) & (st == 1)), (0, "abs"): np.sum((nd == 0) & (st == 2)),
            (1, "esc"): np.sum((nd == 1) & (st == 1)), (1, "abs"): np.sum((nd == 1) & (st == 2)),
            ("2+", None): np.sum(nd >= 2)}


def _z(obs, probs, n):
    """Largest binomial z-score over the categories."""
    return max(abs(obs[c] / n - probs[c]) / np.sqrt(probs[c] * (1 - probs[c]) / n) for c in CATS)


def _check(obs, n, P0, I1, P0_flip, I1_flip, albedo):
    assert sum(obs.values()) == n
    z = _z(obs, A.dust_event_order_probabilities(P0, I1, albedo), n)
    assert z < 4.5, z
    # power: the data reject a reversed albedo test and a mirrored HG angle
    assert _z(obs, A.dust_event_order_probabilities(P0, I1, 1.0 - albedo), n) > 10.0
    assert _z(obs, A.dust_event_order_probabilities(P0_flip, I1_flip, albedo), n) > 10.0


@pytest.mark.parametrize("tau_d,albedo,g", [(1.0, 0.6, 0.73), (2.0, 0.32, 0.5)])
def test_dust_sphere_scattering_orders(orc, tau_d, albedo, g):
    """Dust-only sphere (no HI opacity), central source: the shell transport's albedo branch
    and dust scattering."""
    n = 200000
    r = orc.run_shell(tau0=0.0, T=1e4, R_in=0.0, tau_dust=tau_d, albedo=albedo, g_hg=g, n_photons=n, seed=41,
                      raw=True)
    assert r["n_escaped"] + r["n_absorbed"] == n
    assert int(r["ndust"].sum()) == r["sum_dust_scat"] and r["sum_scat"] == 0
    P0, I1 = A.dust_sphere_first_orders(tau_d, g)
    _, I1f = A.dust_sphere_first_orders(tau_d, -g)
    _check(_observed(r["ndust"], r["status"]), n, P0, I1, P0, I1f, albedo)


def test_dust_cube_scattering_orders(orc):
    """Uniform dusty grid whose HI has no opacity (n_HI = 1e-30 cm^-3 only marks the
    emitting gas, uniformly): the grid transport's albedo branch, cell walk and dust
    scattering, against the Sobol quadrature of the same first orders."""
    side, tau_side, albedo, g = 12, 1.5, 0.6, 0.73
    cell = 3.086e18
    shape = (side,) * 3
    f = {"n_HI": np.full(shape, 1e-30, np.float32), "T": np.full(shape, 1e4, np.float32),
         "vx": np.zeros(shape, np.float32), "vy": np.zeros(shape, np.float32), "vz": np.zeros(shape, np.float32),
         "kd": np.full(shape, tau_side / side / cell, np.float32)}
    n = 120000
    r = orc.run_grid(f, cell_cm=cell, n_photons=n, seed=43, albedo=albedo, g_hg=g, n_bins=8, peel=False, raw=True)
    assert r["sum_scat"] == 0 and int(r["ndust"].sum()) == r["sum_dust_scat"]
    kappa = float(np.float32(tau_side / side / cell)) * cell  # per cell length, as the oracle reads it
    P0, I1 = A.dust_cube_first_orders(kappa, side, g)
    _, I1f = A.dust_cube_first_orders(kappa, side, -g)
    _check(_observed(r["ndust"], r["status"]), n, P0, I1, P0, I1f, albedo)
