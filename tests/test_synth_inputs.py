"""The seeded synthetic inputs (`synth.py`) against the recipes they stand for: the
distributions, scales and structure each workload states (lognormal densities with a given
mean and width, the temperature-density relation of the forest, Gaussian random velocity
fields with a k^-11/3 power spectrum scaled to a per-axis r.m.s., the shell-stream parameter
ranges, the forest's cell scale at z = 2 in the paper's cosmology), and their seeding."""
import numpy as np
import pytest

from paper_2507_11603_gb300 import synth


def test_hubble_and_forest_cell_scale():
    # Planck 2015 (H0 = 67.74, Omega_m = 0.3089): H(z = 2) = 203.6 km/s/Mpc, so a 2 km/s cell
    # is 9.82 proper kpc
    assert synth.hubble(0.0) == pytest.approx(67.74, rel=1e-12)
    assert synth.hubble(2.0) == pytest.approx(67.74 * np.sqrt(0.3089 * 27 + 0.6911), rel=1e-12)
    assert synth.hubble(2.0) == pytest.approx(203.6, abs=0.05)
    assert synth.forest_scale(2.0, 2.0) / (synth.MPC_CM * 1e-3) == pytest.approx(9.824, abs=2e-3)


def test_shell_stream_recipe():
    reqs = synth.shell_stream(4096, seed=2)
    logN = np.log10([r["N_HI"] for r in reqs])
    logT = np.log10([r["T"] for r in reqs])
    v = np.array([r["v_max"] for r in reqs])
    td = np.array([r["tau_dust"] for r in reqs])
    p = np.array([r["n_photons"] for r in reqs], dtype=float)
    assert logN.min() >= 17.0 and logN.max() <= 21.0 and abs(logN.mean() - 19.0) < 0.1
    assert logT.min() >= 3.0 and logT.max() <= 5.0 and abs(logT.mean() - 4.0) < 0.05
    assert v.min() >= 0.0 and v.max() <= 500.0 and abs(v.mean() - 250.0) < 10.0
    assert td.min() >= 0.0 and td.max() <= 2.0 and abs(td.mean() - 1.0) < 0.04
    assert p.min() >= 1e3 and p.max() <= 1e5
    # log-uniform photon counts on [1e3, 1e5]: mean (1e5 - 1e3) / ln 100 = 2.15e4
    assert p.mean() == pytest.approx((1e5 - 1e3) / np.log(100.0), rel=0.05)
    assert len({r["seed"] for r in reqs}) == len(reqs)
    # the default stream is the first 256 requests of the same draw order, and seeded
    first = synth.shell_stream(256, seed=2)
    assert first == synth.shell_stream(256, seed=2)
    assert np.log10(max(r["N_HI"] for r in synth.shell_stream(256, seed=2, nhi_max=1e19))) <= 19.0
    # Poisson arrivals: exponential gaps at the given rate, the first request at t = 0
    t = np.array([r["arrival_s"] for r in synth.shell_stream(4096, seed=3, rate_hz=20.0)])
    gaps = np.diff(t)
    assert t[0] == 0.0 and np.all(gaps >= 0) and gaps.mean() == pytest.approx(0.05, rel=0.06)


def _radial_power_slope(f, kmin=3, kmax=12):
    n = f.shape[0]
    P = np.abs(np.fft.rfftn(f)) ** 2
    k = [np.fft.fftfreq(n) * n for _ in range(f.ndim - 1)] + [np.fft.rfftfreq(n) * n]
    kk = np.sqrt(sum(np.meshgrid(*[ki ** 2 for ki in k], indexing="ij")))
    bins = np.arange(kmin, kmax + 1)
    kc, Pc = [], []
    for lo, hi in zip(bins[:-1], bins[1:]):
        m = (kk >= lo) & (kk < hi)
        kc.append(kk[m].mean())
        Pc.append(P[m].mean())
    return np.polyfit(np.log(kc), np.log(Pc), 1)[0]


def test_grid_fields_recipe():
    f = synth.grid_fields(n=48, seed=3)
    n = f["n_HI"].astype(np.float64)
    lnn = np.log(n)
    # lognormal n_HI: mean 1e-3 cm^-3 (the mean of n, mu_ln = ln(mean) - sigma^2 / 2), sigma_ln 1.5
    assert lnn.std() == pytest.approx(1.5, rel=0.01)
    assert lnn.mean() == pytest.approx(np.log(1e-3) - 0.5 * 1.5 ** 2, abs=0.02)
    assert n.mean() == pytest.approx(1e-3, rel=0.1)
    # lognormal T around a 1e4 K median, sigma_ln 0.5
    lnT = np.log(f["T"].astype(np.float64))
    assert np.median(lnT) == pytest.approx(np.log(1e4), abs=0.02) and lnT.std() == pytest.approx(0.5, rel=0.01)
    # three velocity components: zero mean, 50 km/s r.m.s. each, uncorrelated, P(k) ~ k^-11/3
    v = f["v"].astype(np.float64)
    assert v.shape == (3, 48, 48, 48)
    for c in range(3):
        assert abs(v[c].mean()) < 1e-3 and v[c].std() == pytest.approx(50.0, rel=1e-4)
        assert _radial_power_slope(v[c]) == pytest.approx(-11.0 / 3.0, abs=0.25)
    # independent components: the real-space correlation of k^-11/3 fields is dominated by a
    # few large-scale modes, so compare the modes whitened by the spectrum (each mode counts once)
    kk = np.sqrt(sum(k ** 2 for k in np.meshgrid(np.fft.fftfreq(48), np.fft.fftfreq(48), np.fft.rfftfreq(48),
                                                indexing="ij")))
    m = kk > 0
    w = [np.fft.rfftn(v[c])[m] * kk[m] ** (11.0 / 6.0) for c in range(3)]
    for a, b in ((0, 1), (0, 2), (1, 2)):
        ca = np.concatenate([w[a].real, w[a].imag])
        cb = np.concatenate([w[b].real, w[b].imag])
        assert abs(np.corrcoef(ca, cb)[0, 1]) < 0.02
    # dust extinction 0.01 n_HI sigma_dust
    assert np.allclose(f["kd"], (0.01 * n * 4e-22).astype(np.float32), rtol=1e-6, atol=0)
    # seeded
    g = synth.grid_fields(n=48, seed=3)
    assert all(np.array_equal(f[k], g[k]) for k in f)
    assert not np.array_equal(f["n_HI"], synth.grid_fields(n=48, seed=4)["n_HI"])


def test_forest_fields_recipe():
    nHI, T, v = synth.forest_fields_numpy((32, 32, 32), seed=5)
    ratio = nHI.astype(np.float64) / 1e-10
    # lognormal (mean 1e-10, sigma_ln 2) and T = 1e4 (1 + delta)^0.6 with 1 + delta = n / <n>
    assert np.log(ratio).std() == pytest.approx(2.0, rel=0.02)
    assert np.log(ratio).mean() == pytest.approx(-2.0, abs=0.05)
    assert np.allclose(T, (1e4 * ratio ** 0.6).astype(np.float32), rtol=1e-5)
    assert abs(v.mean()) < 1e-3 and v.astype(np.float64).std() == pytest.approx(30.0, rel=1e-4)
    assert _radial_power_slope(v.astype(np.float64), kmin=2, kmax=9) == pytest.approx(-11.0 / 3.0, abs=0.3)


def test_forest_fields_torch_recipe_on_cpu():
    """The generator of the full box (torch, FP32) follows the same recipe; run here on the
    CPU on a box of 1024-cell columns."""
    torch = pytest.importorskip("torch")
    nHI, T, v = synth.forest_fields_torch(seed=5, device="cpu", shape=(1024, 8, 8))
    assert tuple(nHI.shape) == (1024, 8, 8)
    ratio = nHI.double() / 1e-10
    assert float(torch.log(ratio).std()) == pytest.approx(2.0, rel=0.02)
    assert torch.allclose(T.double(), 1e4 * ratio ** 0.6, rtol=1e-4)
    assert float(v.double().std()) == pytest.approx(30.0, rel=1e-3) and abs(float(v.double().mean())) < 1e-2
