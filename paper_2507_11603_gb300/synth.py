"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws random fields and
request lists (numpy / torch random generators), which both the CUDA path and the
FP64 oracle then consume as plain arrays.

Recipes (the paper's own inputs -- TNG50, GIBLE, MCST snapshots, the Faucher-Giguere
et al. 2010 comparison runs -- are not available; these stand in for them):
  * shell stream: log-uniform N_HI in [1e17, 1e21] cm^-2, log-uniform T in
    [1e3, 1e5] K, uniform v_max in [0, 500] km/s, uniform tau_d in [0, 2],
    log-uniform photon counts in [1e3, 1e5], Poisson arrivals (Sec. 5.1 shell grid);
  * grid: n_HI lognormal (given mean, sigma_ln), T lognormal around its median,
    three independent Gaussian random velocity fields with P(k) ~ k^-11/3 scaled to a
    per-axis sigma (k = 0 mode removed, periodic), dust extinction proportional to n_HI;
  * forest: n_HI lognormal (mean, sigma_ln), T = T0 (1 + delta)^0.6 with
    1 + delta = n_HI / <n_HI>, v_los a Gaussian random field with the same spectrum.
"""
from __future__ import annotations

import numpy as np

# Planck 2015 cosmology used by the paper (Sec. 5 footnote): H(z) for the forest scale.
H0 = 67.74  # km/s/Mpc
OMEGA_M, OMEGA_L = 0.3089, 0.6911
MPC_CM = 3.0856775814913673e24
PC_CM = 3.0856775814913673e18


def hubble(z: float) -> float:
    """H(z) in km/s/Mpc."""
    return H0 * np.sqrt(OMEGA_M * (1 + z) ** 3 + OMEGA_L)


def forest_scale(z: float = 2.0, dv_cell: float = 2.0) -> float:
    """Proper path length [cm] of one cell whose Hubble velocity width is dv_cell."""
    return dv_cell / hubble(z) * MPC_CM


def shell_stream(n: int = 256, seed: int = 2, rate_hz: float | None = None, nhi_max: float = 1e21):
    rng = np.random.default_rng(seed)
    logN = rng.uniform(17.0, np.log10(nhi_max), n)
    logT = rng.uniform(3.0, 5.0, n)
    v = rng.uniform(0.0, 500.0, n)
    tau_d = rng.uniform(0.0, 2.0, n)
    logp = rng.uniform(3.0, 5.0, n)
    reqs = []
    for i in range(n):
        reqs.append({"N_HI": float(10 ** logN[i]), "T": float(10 ** logT[i]), "v_max": float(v[i]),
                     "tau_dust": float(tau_d[i]), "n_photons": int(round(10 ** logp[i])), "seed": (2 << 32) | i})
    if rate_hz:
        gaps = rng.exponential(1.0 / rate_hz, n)
        t = np.cumsum(gaps) - gaps[0]
    else:
        t = np.zeros(n)
    for r, ti in zip(reqs, t):
        r["arrival_s"] = float(ti)
    return reqs


def _grf_numpy(shape, sigma, rng, index=-11.0 / 3.0):
    white = rng.standard_normal(shape)
    f = np.fft.rfftn(white)
    k = [np.fft.fftfreq(n) for n in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    kk = np.sqrt(sum(np.meshgrid(*[ki ** 2 for ki in k], indexing="ij", sparse=True)))
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (index / 2.0)
    f *= amp
    g = np.fft.irfftn(f, s=shape, axes=tuple(range(len(shape))))
    g -= g.mean()
    return (g * (sigma / g.std())).astype(np.float32)


def grid_fields(n: int = 256, seed: int = 3, mean_nHI: float = 1e-3, sigma_ln: float = 1.5, T_med: float = 1e4,
                sigma_lnT: float = 0.5, sigma_v: float = 50.0, dust_ratio: float = 0.01,
                sigma_dust: float = 4e-22):
    """Fields of shape (n, n, n) float32; v of shape (3, n, n, n); kd = dust extinction [cm^-1]
    = dust_ratio * n_HI * sigma_dust (sigma_dust: per-H extinction cross-section at Lya)."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    nHI = (mean_nHI * np.exp(sigma_ln * rng.standard_normal(shape) - 0.5 * sigma_ln ** 2)).astype(np.float32)
    T = (T_med * np.exp(sigma_lnT * rng.standard_normal(shape))).astype(np.float32)
    v = np.stack([_grf_numpy(shape, sigma_v, rng) for _ in range(3)])
    kd = (dust_ratio * nHI.astype(np.float64) * sigma_dust).astype(np.float32)
    return {"n_HI": nHI, "T": T, "v": np.ascontiguousarray(v), "kd": kd}


def forest_fields_numpy(shape, seed: int = 5, mean_nHI: float = 1e-10, sigma_ln: float = 2.0, T0: float = 1e4,
                        sigma_v: float = 30.0):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(shape)
    ratio = np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2)
    nHI = (mean_nHI * ratio).astype(np.float32)
    T = (T0 * ratio ** 0.6).astype(np.float32)
    v = _grf_numpy(shape, sigma_v, rng)
    return nHI, T, v


def forest_fields_torch(n: int = 1024, seed: int = 5, mean_nHI: float = 1e-10, sigma_ln: float = 2.0,
                        T0: float = 1e4, sigma_v: float = 30.0, device: str = "cuda", shape=None):
    """The 1024^3 forest box generated on the GPU in FP32 (torch.fft), fields (nz, ny, nx);
    `shape` = (nz, ny, nx) for a box of other proportions (e.g. fewer sightlines of the
    full 1024 cells)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    shape = tuple(shape) if shape is not None else (n, n, n)
    g = torch.randn(shape, generator=gen, device=device, dtype=torch.float32)
    ratio = torch.exp(sigma_ln * g - 0.5 * sigma_ln ** 2)
    del g
    nHI = (mean_nHI * ratio).float()
    T = (T0 * ratio.pow(0.6)).float()
    del ratio
    w = torch.randn(shape, generator=gen, device=device, dtype=torch.float32)
    f = torch.fft.rfftn(w)
    del w
    kz = torch.fft.fftfreq(shape[0], device=device)
    ky = torch.fft.fftfreq(shape[1], device=device)
    kx = torch.fft.rfftfreq(shape[2], device=device)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    amp = torch.where(k2 > 0, k2.clamp_min(1e-30).pow(-11.0 / 12.0), torch.zeros_like(k2))
    f *= amp
    del amp, k2
    v = torch.fft.irfftn(f, s=shape)
    del f
    v -= v.mean()
    v *= sigma_v / v.std()
    return nHI.contiguous(), T.contiguous(), v.float().contiguous()
