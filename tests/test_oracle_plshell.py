"""Pins of the oracle's power-law shells and post-processing reweighting (Sec. 5.1)."""
import numpy as np
import pytest
from scipy import integrate, stats


def test_profiles_are_normalised(orc):
    # radial HI column between the radii = N_HI (tau0 = N_HI sigma_0), distance-averaged
    # outflow speed = v_avg, for several power-law indices
    sig0 = orc.line_params(1e4)["sigma0"]
    for ar, av, dv in [(0.0, 1.0, 10.0), (-0.5, 0.5, 3.0), (-1.0, 1.5, 20.0), (-2.0, 0.0, 1.5)]:
        ri = 1.0 / dv
        kw = dict(dv_ratio=dv, N_HI=1e18, T=1e4, v_avg=120.0, alpha_rho=ar, alpha_v=av)
        col = integrate.quad(lambda r: orc.plshell_profile(r=r, **kw)[0], ri, 1.0, epsrel=1e-11)[0]
        vav = integrate.quad(lambda r: orc.plshell_profile(r=r, **kw)[1], ri, 1.0, epsrel=1e-11)[0] / (1 - ri)
        assert abs(col / (1e18 * sig0) - 1) < 1e-9
        assert abs(vav / 120.0 - 1) < 1e-9
        k1, v1 = orc.plshell_profile(r=1.0, **kw)
        k2, v2 = orc.plshell_profile(r=0.5 * (1 + ri), **kw)
        assert abs(k2 / k1 - (0.5 * (1 + ri)) ** ar) < 1e-12 and abs(v2 / v1 - (0.5 * (1 + ri)) ** av) < 1e-12


def test_homologous_uniform_case_equals_the_linear_shell(orc):
    # alpha_rho = 0, alpha_v = 1 is the uniform shell with v = v_max r (pinned elsewhere);
    # the general path integrates a different representation of the same x(s), so the same
    # stream must give the same photons
    sig0 = orc.line_params(1e4)["sigma0"]
    n = 400
    v_max = 200.0
    kw = dict(n_photons=n, seed=3, n_bins=50, X_min=-1500.0, X_max=1500.0)
    a = orc.run_shell(tau0=1e17 * sig0, T=1e4, R_in=0.9, v_max=v_max, tau_dust=0.3, phase="dipole",
                      line="gauss", sigma=50.0, raw=True, **kw)
    b = orc.run_plshell(dv_ratio=1 / 0.9, N_HI=1e17, T=1e4, v_avg=0.95 * v_max, alpha_rho=0.0, alpha_v=1.0,
                        tau_dust=0.3, phase="dipole", sigma=50.0, ew=0.0, C_cont=0.0, **kw)
    same = (a["status"] == b["status"]) & (np.abs(a["X"] - b["X"]) < 1e-6)
    assert same.mean() > 0.99, same.mean()


def test_free_streaming_records(orc):
    # no gas to speak of: photons escape radially with X = X0 and cross exactly one radial column
    r = orc.run_plshell(dv_ratio=5.0, N_HI=1e8, T=1e4, v_avg=100.0, alpha_rho=-1.0, alpha_v=0.5,
                        sigma=300.0, ew=500.0, C_cont=2000.0, n_photons=300, seed=5)
    assert (r["status"] == 1).all() and (r["nscat"] == 0).all()
    assert np.array_equal(r["X"], r["X0"])
    assert np.abs(r["col"] - 1.0).max() < 1e-9


def test_intrinsic_spectrum_sampling(orc):
    # X0 follows p(X) = pl N(0, sigma^2) + (1 - pl) U(-C, C), pl = ew / (ew + 2C)
    sigma, ew, Cc = 300.0, 740.0, 2500.0
    r = orc.run_plshell(dv_ratio=5.0, N_HI=1e8, T=1e4, v_avg=100.0, sigma=sigma, ew=ew, C_cont=Cc,
                        n_photons=20000, seed=6)
    pl = ew / (ew + 2 * Cc)

    def cdf(x):
        return pl * stats.norm.cdf(x, scale=sigma) + (1 - pl) * np.clip((x + Cc) / (2 * Cc), 0, 1)
    assert stats.kstest(r["X0"], cdf).pvalue > 1e-3


def test_reweight_identity_and_dust(orc):
    samp = (800.0, 740.0, 2500.0)
    kw = dict(dv_ratio=10.0, N_HI=10 ** 17.6, T=1e4, v_avg=120.0, alpha_rho=-0.5, alpha_v=1.0, sigma=samp[0],
              ew=samp[1], C_cont=samp[2], n_bins=40, X_min=-2000.0, X_max=2000.0, n_photons=6000)
    clean = orc.run_plshell(seed=7, **kw)
    # target = sampled spectrum, no dust: every weight is 1
    w = orc.reweight(clean["X0"], clean["X"], clean["col"], clean["status"], sample=samp, target=samp, tau_d=0.0,
                     n_bins=40, X_min=-2000.0, X_max=2000.0)
    assert np.allclose(w[:40] * 6000, clean["counts"], rtol=0, atol=1e-9)
    # dust following the gas in the transport == dust-free run reweighted by exp(-tau_d col)
    tau_d = 0.8
    dusty = orc.run_plshell(seed=8, tau_dust=tau_d, **kw)
    rw = orc.reweight(clean["X0"], clean["X"], clean["col"], clean["status"], sample=samp, target=samp,
                      tau_d=tau_d, n_bins=40, X_min=-2000.0, X_max=2000.0)
    f_rt = dusty["n_escaped"] / 6000
    f_rw = rw.sum()
    assert abs(f_rt - f_rw) < 4 * np.sqrt(f_rt * (1 - f_rt) / 6000), (f_rt, f_rw)
    # per-bin: binomial counts vs weighted sums
    c = dusty["counts"] / 6000.0
    var = c / 6000.0 + rw[:40] / 6000.0
    m = (c + rw[:40]) > 5.0 / 6000
    chi2 = np.sum((c[m] - rw[:40][m]) ** 2 / var[m]) / m.sum()
    assert chi2 < 2.0, chi2


def test_mgii_line_data(orc):
    """Mg II doublet data: thermal speed scales as sqrt(m_H / m_Mg) from the HI value, the
    line-centre cross-sections are in the ratio f_K lambda_K : f_H lambda_H, and the H line
    sits c (lambda_K / lambda_H - 1) = -767.68 km/s from K."""
    m = orc.mgii_params(1e4)
    h = orc.line_params(1e4)
    assert abs(m["vth_kms"] / h["vth_kms"] - np.sqrt(1.6735575e-24 / (24.305 * 1.66053906660e-24))) < 1e-12
    assert abs(m["sigma0_K"] / m["sigma0_H"] - (0.608 * 2796.352) / (0.303 * 2803.531)) < 1e-12
    assert abs(m["X_H"] - 299792.458 * (2796.352 / 2803.531 - 1.0)) < 1e-9
    assert 2.1e-3 < m["a_K"] < 2.3e-3 and 2.1e-3 < m["a_H"] < 2.3e-3


@pytest.mark.parametrize("where", ["K", "H", "between"])
def test_mgii_first_flight_escape(orc, where):
    """Static uniform sphere around a monochromatic source: the fraction of photons that
    escape without scattering is exp(-tau(X)), tau summed over both transitions, each with
    its own Voigt profile (scipy's Faddeeva function) at its own offset."""
    from scipy.special import wofz
    m = orc.mgii_params(1e4)
    X0 = {"K": 0.0, "H": m["X_H"], "between": 0.5 * m["X_H"]}[where]
    N = 1.5e12
    n = 20000
    r = orc.run_plshell(dv_ratio=1000.0, N_HI=N, T=1e4, v_avg=0.0, alpha_rho=0.0, alpha_v=1.0, phase="dipole",
                        sigma=1e-4, ew=1.0, C_cont=0.0, X0=X0, n_photons=n, seed=11, species="MgII")
    xK = X0 / m["vth_kms"]
    xH = (X0 + (2803.531 / 2796.352 - 1.0) * (299792.458 + X0)) / m["vth_kms"]
    tau = N * (m["sigma0_K"] * wofz(xK + 1j * m["a_K"]).real
                            + m["sigma0_H"] * wofz(xH + 1j * m["a_H"]).real)
    p = np.exp(-tau)
    f = float(np.mean(r["nscat"] == 0))
    assert abs(f - p) < 4 * np.sqrt(max(p * (1 - p), 1e-9) / n) + 1e-9, (where, f, p, tau)


def test_power_law_first_flight_escape(orc):
    """A monochromatic central source in a power-law shell (n ~ r^-1, v ~ r^0.5, dust
    following the gas): the fraction of photons that escape without any interaction is
    exp(-tau_HI(X0) - tau_d), with tau_HI = int k(r) H(a, (X0 - v(r)) / v_th) dr along the
    radial ray, by scipy quadrature of the shell's profiles and scipy's Faddeeva function."""
    from scipy.special import wofz
    lp = orc.line_params(1e4)
    kw = dict(dv_ratio=5.0, N_HI=3e14, T=1e4, v_avg=150.0, alpha_rho=-1.0, alpha_v=0.5)
    tau_d, n = 0.3, 20000

    def tau_hi(X0):
        def f(r):
            k, v = orc.plshell_profile(r=r, **kw)
            return k * wofz((X0 - v) / lp["vth_kms"] + 1j * lp["a"]).real
        return integrate.quad(f, 1.0 / kw["dv_ratio"], 1.0, limit=400, epsabs=0, epsrel=1e-9)[0]

    for X0 in (100.0, 120.0, 160.0, 200.0, 240.0):
        t = tau_hi(X0)
        r = orc.run_plshell(**kw, tau_dust=tau_d, phase="dipole", sigma=1e-4, ew=1.0, C_cont=0.0, X0=X0,
                            n_photons=n, seed=13)
        f = float(np.mean((r["status"] == 1) & (r["nscat"] == 0)))
        p = np.exp(-t - tau_d)
        assert abs(f - p) < 4 * np.sqrt(p * (1 - p) / n), (X0, t, f, p)
