"""FP64 CPU oracle for the resonant Lyman-alpha Monte Carlo hot path (THOR,
arXiv:2507.11603).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm may import this package.  The CUDA
product path never imports it, and it never imports the product path.  Inputs
come in as plain arrays drawn by the seeded generators of the synthetic-input
module, which holds none of the method's arithmetic.

The arithmetic is in ``thor_oracle.cpp`` (plain C++17, double precision); this
module compiles it with g++ and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "thor_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++, -O2, no FMA contraction: the DDA contract is bit-exact)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Line(C.Structure):
    _fields_ = [("vth_kms", C.c_double), ("a", C.c_double), ("sigma0", C.c_double)]


class Shell(C.Structure):
    """Gridless geometry (Sec. 3.3): shell/sphere (geometry 0) or slab (geometry 1)."""
    _fields_ = [("geometry", C.c_int32), ("phase", C.c_int32), ("core_skip", C.c_int32), ("pad", C.c_int32),
                ("R_in", C.c_double), ("R_out", C.c_double), ("tau0", C.c_double),
                ("T", C.c_double), ("v_max", C.c_double), ("tau_dust", C.c_double),
                ("albedo", C.c_double), ("g_hg", C.c_double)]


class Source(C.Structure):
    _fields_ = [("line", C.c_int32), ("pad", C.c_int32), ("X0", C.c_double), ("sigma", C.c_double)]


class Result(C.Structure):
    _fields_ = [("n_escaped", C.c_uint64), ("n_absorbed", C.c_uint64), ("n_capped", C.c_uint64),
                ("sum_scat", C.c_uint64), ("sum_scat2", C.c_double), ("sum_dust_scat", C.c_uint64),
                ("sum_upar_iters", C.c_uint64), ("unused", C.c_double)]


class PLShell(C.Structure):
    """Power-law shell of the shell-model sweep (Sec. 5.1)."""
    _fields_ = [("dv_ratio", C.c_double), ("N_HI", C.c_double), ("T", C.c_double), ("v_avg", C.c_double),
                ("alpha_rho", C.c_double), ("alpha_v", C.c_double), ("tau_dust", C.c_double),
                ("phase", C.c_int32), ("species", C.c_int32)]


SPECIES = {"HI": 0, "MgII": 1}


class PLSource(C.Structure):
    _fields_ = [("sigma", C.c_double), ("ew", C.c_double), ("C", C.c_double), ("X0", C.c_double)]


class GridRun(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("phase", C.c_int32), ("cell_cm", C.c_double),
                ("albedo", C.c_double), ("g_hg", C.c_double), ("n_bins", C.c_int32),
                ("img_nx", C.c_int32), ("X_min", C.c_double), ("X_max", C.c_double),
                ("peel", C.c_int32), ("pad", C.c_int32), ("max_scat", C.c_uint64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.POINTER
            L.orc_line_params.argtypes = [C.c_double, P(Line)]
            L.orc_philox.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            L.orc_stream_words.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, P(C.c_uint32)]
            L.orc_dawson.restype = C.c_double
            L.orc_dawson.argtypes = [C.c_double]
            L.orc_voigt.restype = C.c_double
            L.orc_voigt.argtypes = [C.c_double, C.c_double]
            L.orc_voigt_batch.argtypes = [P(C.c_double), P(C.c_double), P(C.c_double), C.c_int64]
            L.orc_u0.restype = C.c_double
            L.orc_u0.argtypes = [C.c_double, C.c_double]
            L.orc_u0_eq10.restype = C.c_double
            L.orc_u0_eq10.argtypes = [C.c_double, C.c_double]
            L.orc_eq10_mass.restype = C.c_double
            L.orc_eq10_mass.argtypes = [C.c_double, C.c_double, C.c_double]
            L.orc_set_upar_method.argtypes = [C.c_int]
            L.orc_xcw.restype = C.c_double
            L.orc_xcw.argtypes = [C.c_double]
            L.orc_get_upar_method.restype = C.c_int
            L.orc_segment_tau.restype = C.c_double
            L.orc_segment_tau.argtypes = [C.c_double] * 7 + [P(C.c_double)]
            L.orc_sample_upar.argtypes = [C.c_double, C.c_double, C.c_uint64, C.c_int64,
                                          P(C.c_double), P(C.c_uint64)]
            L.orc_sample_mu.argtypes = [C.c_int, C.c_double, C.c_uint64, C.c_int64, P(C.c_double)]
            L.orc_scatter_once.argtypes = [C.c_double, C.c_double, C.c_int, C.c_uint64, C.c_int64,
                                           P(C.c_double), P(C.c_double)]
            L.orc_run_shell.restype = C.c_int
            L.orc_run_shell.argtypes = [P(Shell), P(Source), C.c_uint64, C.c_uint64, C.c_uint64,
                                        C.c_int32, C.c_double, C.c_double, C.c_uint64, C.c_int32,
                                        P(C.c_uint64), P(Result), P(C.c_double), P(C.c_uint64),
                                        P(C.c_uint8), P(C.c_uint32)]
            L.orc_plshell_profile.argtypes = [P(PLShell), C.c_double, P(C.c_double), P(C.c_double)]
            L.orc_mgii_params.argtypes = [C.c_double, P(C.c_double)]
            L.orc_run_plshell.restype = C.c_int
            L.orc_run_plshell.argtypes = [P(PLShell), P(PLSource), C.c_uint64, C.c_uint64, C.c_uint64,
                                          C.c_int32, C.c_double, C.c_double, C.c_uint64, C.c_int32,
                                          P(C.c_uint64), P(Result), P(C.c_double), P(C.c_double),
                                          P(C.c_double), P(C.c_uint64), P(C.c_uint8)]
            L.orc_reweight.argtypes = [C.c_int64, P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_uint8)] + \
                [C.c_double] * 7 + [C.c_int32, C.c_double, C.c_double, P(C.c_double)]
            L.orc_dda_trace.restype = C.c_int
            L.orc_dda_trace.argtypes = [P(C.c_int32), P(C.c_double), P(C.c_float), C.c_int32,
                                        C.c_int32, P(C.c_int64), P(C.c_double), P(C.c_int32)]
            L.orc_run_grid.restype = C.c_int
            L.orc_run_grid.argtypes = [P(C.c_float)] * 6 + [P(GridRun), C.c_uint64, C.c_uint64,
                                                             C.c_uint64, C.c_int32, P(C.c_uint64),
                                                             P(C.c_double), P(Result), P(C.c_double),
                                                             P(C.c_uint64), P(C.c_uint8), P(C.c_double),
                                                             P(C.c_uint32)]
            L.orc_forest.restype = C.c_int
            L.orc_forest.argtypes = [P(C.c_float)] * 3 + [C.c_int32] * 3 + [P(C.c_int32), P(C.c_int32),
                                                                            C.c_int32, C.c_double,
                                                                            C.c_double, C.c_int32,
                                                                            C.c_double, C.c_int32,
                                                                            P(C.c_double)]
            _lib = L
    return _lib


def _p(arr, ctype):
    return arr.ctypes.data_as(C.POINTER(ctype))


# Exact u_par samplers of the oracle (Sec. 3.4, Eq. 10).  "eq10" (the default) is the
# two-piece comparison function as printed, with its split point chosen by minimising the
# envelope mass; "envelope" is a three-piece variant that reads the random words exactly as
# the CUDA sampler does, for tests that follow the same photon on both sides draw by draw.
UPAR_SAMPLERS = {"envelope": 0, "eq10": 1}
_sampler_lock = threading.RLock()


class _sampler:
    """Selects the oracle's u_par sampler for the duration of one call."""

    def __init__(self, name: str):
        if name not in UPAR_SAMPLERS:
            raise ValueError(f"unknown u_par sampler {name!r}")
        self.m = UPAR_SAMPLERS[name]

    def __enter__(self):
        _sampler_lock.acquire()
        self.prev = lib().orc_get_upar_method()
        lib().orc_set_upar_method(self.m)

    def __exit__(self, *exc):
        lib().orc_set_upar_method(self.prev)
        _sampler_lock.release()


# ---------------------------------------------------------------------------------
# Line physics and special functions
# ---------------------------------------------------------------------------------
def line_params(T: float) -> dict:
    """v_th [km/s], Voigt parameter a and sigma_0 [cm^2] at temperature T (Sec. 2.3.1)."""
    out = Line()
    lib().orc_line_params(float(T), C.byref(out))
    return {"vth_kms": out.vth_kms, "a": out.a, "sigma0": out.sigma0}


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(o, C.c_uint32))
    return o


def stream_words(seed: int, photon: int, n: int) -> np.ndarray:
    o = np.zeros(n, dtype=np.uint32)
    lib().orc_stream_words(seed, photon, n, _p(o, C.c_uint32))
    return o


def dawson(x: float) -> float:
    return lib().orc_dawson(float(x))


def voigt(a, x) -> np.ndarray:
    """H(a,x) = Re w(x + i a) in double precision (App. A.3 truth)."""
    a_, x_ = np.broadcast_arrays(np.asarray(a, dtype=np.float64), np.asarray(x, dtype=np.float64))
    a_ = np.ascontiguousarray(a_.ravel())
    x_ = np.ascontiguousarray(x_.ravel())
    o = np.empty_like(x_)
    lib().orc_voigt_batch(_p(a_, C.c_double), _p(x_, C.c_double), _p(o, C.c_double), o.size)
    return o.reshape(np.broadcast(np.asarray(a), np.asarray(x)).shape)


def xcw(a: float) -> float:
    """Core-to-wing transition x_cw(a) of the Voigt profile (App. A.2), exact (Newton)."""
    return lib().orc_xcw(float(a))


def u0_rule(x: float, a: float) -> float:
    """Split point u0 of the three-piece ("envelope") sampler."""
    return lib().orc_u0(float(x), float(a))


def u0_eq10(x: float, a: float) -> float:
    """Split point u0 of the two-piece Eq. 10 sampler: the minimiser of its envelope mass."""
    return lib().orc_u0_eq10(float(x), float(a))


def eq10_envelope_mass(x: float, a: float, u0: float) -> float:
    """Mass of the two-piece Eq. 10 comparison function times a."""
    return lib().orc_eq10_mass(float(x), float(a), float(u0))


def segment_tau(x0, gam, kap0, kapd, a, S, tau_rem=np.inf):
    """Total tau over a linear-drift segment, or the crossing point if tau_rem is reached."""
    s = C.c_double()
    tt = lib().orc_segment_tau(x0, gam, kap0, kapd, a, S, float(tau_rem), C.byref(s))
    return tt, s.value


# ---------------------------------------------------------------------------------
# Samplers (unit level)
# ---------------------------------------------------------------------------------
def sample_upar(x: float, a: float, n: int, seed: int = 0, sampler: str = "eq10"):
    o = np.empty(n)
    it = C.c_uint64()
    with _sampler(sampler):
        lib().orc_sample_upar(float(x), float(a), seed, n, _p(o, C.c_double), C.byref(it))
    return o, it.value


def sample_mu(kind: str, n: int, g: float = 0.0, seed: int = 0) -> np.ndarray:
    k = {"isotropic": 0, "dipole": 1, "hg": 2}[kind]
    o = np.empty(n)
    lib().orc_sample_mu(k, float(g), seed, n, _p(o, C.c_double))
    return o


def scatter_once(x_in: float, a: float, phase: int, n: int, seed: int = 0, sampler: str = "eq10"):
    xo = np.empty(n)
    mu = np.empty(n)
    with _sampler(sampler):
        lib().orc_scatter_once(float(x_in), float(a), int(phase), seed, n, _p(xo, C.c_double),
                               _p(mu, C.c_double))
    return xo, mu


# ---------------------------------------------------------------------------------
# Transport
# ---------------------------------------------------------------------------------
PHASE = {"isotropic": 0, "dipole": 1, "mixed": 2}


def run_shell(*, tau0, T, R_in=0.0, R_out=1.0, v_max=0.0, tau_dust=0.0, albedo=0.0, g_hg=0.73,
              phase="isotropic", geometry="shell", line="delta", X0=0.0, sigma=0.0,
              n_photons=1000, seed=0, first_id=0, n_bins=200, X_min=-500.0, X_max=500.0,
              max_scat=0, n_threads=0, raw=False, core_skip=False, sampler="eq10"):
    geo = Shell(0 if geometry == "shell" else 1, PHASE[phase], 1 if core_skip else 0, 0, R_in, R_out, tau0, T,
                v_max, tau_dust, albedo, g_hg)
    src = Source(0 if line == "delta" else 1, 0, X0, sigma)
    counts = np.zeros(n_bins + 2, dtype=np.uint64)
    res = Result()
    rx = rn = rs = rd = None
    if raw:
        rx = np.zeros(n_photons)
        rn = np.zeros(n_photons, dtype=np.uint64)
        rs = np.zeros(n_photons, dtype=np.uint8)
        rd = np.zeros(n_photons, dtype=np.uint32)
    with _sampler(sampler):
        rc = lib().orc_run_shell(C.byref(geo), C.byref(src), first_id, n_photons, seed, n_bins, X_min,
                                 X_max, max_scat, n_threads, _p(counts, C.c_uint64), C.byref(res),
                                 _p(rx, C.c_double) if raw else None,
                                 _p(rn, C.c_uint64) if raw else None,
                                 _p(rs, C.c_uint8) if raw else None,
                                 _p(rd, C.c_uint32) if raw else None)
    if rc != 0:
        raise ValueError("orc_run_shell rejected its arguments")
    out = {"counts": counts[:n_bins], "underflow": int(counts[n_bins]), "overflow": int(counts[n_bins + 1]),
           "n_escaped": res.n_escaped, "n_absorbed": res.n_absorbed, "n_capped": res.n_capped,
           "sum_scat": res.sum_scat, "sum_scat2": res.sum_scat2, "sum_dust_scat": res.sum_dust_scat,
           "sum_upar_iters": res.sum_upar_iters}
    if raw:
        out.update(X=rx, nscat=rn, status=rs, ndust=rd)
    return out


def plshell_profile(*, dv_ratio, N_HI, T, v_avg, alpha_rho, alpha_v, r):
    """HI opacity per unit length (outer radius = 1) and outflow speed at radius r."""
    geo = PLShell(dv_ratio, N_HI, T, v_avg, alpha_rho, alpha_v, 0.0, 1, SPECIES["HI"])
    k, v = C.c_double(), C.c_double()
    lib().orc_plshell_profile(C.byref(geo), r, C.byref(k), C.byref(v))
    return k.value, v.value


def mgii_params(T):
    """Mg II doublet line data at T: v_th, a and sigma_0 of K and H, H centre on the K scale."""
    out = np.zeros(6)
    lib().orc_mgii_params(T, _p(out, C.c_double))
    return {"vth_kms": out[0], "a_K": out[1], "sigma0_K": out[2], "a_H": out[3], "sigma0_H": out[4],
            "X_H": out[5]}


def run_plshell(*, dv_ratio, N_HI, T, v_avg, alpha_rho=0.0, alpha_v=1.0, tau_dust=0.0, phase="dipole",
                sigma=800.0, ew=0.0, C_cont=0.0, n_photons=1000, seed=0, first_id=0, n_bins=200,
                X_min=-2500.0, X_max=2500.0, max_scat=0, n_threads=0, species="HI", X0=0.0,
                sampler="eq10"):
    """Power-law shell run (Sec. 5.1) with per-photon records X0, X, col (units of N_HI);
    species "MgII": the doublet, N_HI is then the Mg II column."""
    geo = PLShell(dv_ratio, N_HI, T, v_avg, alpha_rho, alpha_v, tau_dust, PHASE[phase], SPECIES[species])
    src = PLSource(sigma, ew, C_cont, X0)
    counts = np.zeros(n_bins + 2, dtype=np.uint64)
    res = Result()
    x0, x, col = np.zeros(n_photons), np.zeros(n_photons), np.zeros(n_photons)
    rn = np.zeros(n_photons, dtype=np.uint64)
    rs = np.zeros(n_photons, dtype=np.uint8)
    with _sampler(sampler):
        rc = lib().orc_run_plshell(C.byref(geo), C.byref(src), first_id, n_photons, seed, n_bins, X_min,
                                   X_max, max_scat, n_threads, _p(counts, C.c_uint64), C.byref(res),
                                   _p(x0, C.c_double), _p(x, C.c_double), _p(col, C.c_double),
                                   _p(rn, C.c_uint64), _p(rs, C.c_uint8))
    if rc != 0:
        raise ValueError("orc_run_plshell rejected its arguments")
    return {"counts": counts[:n_bins], "underflow": int(counts[n_bins]), "overflow": int(counts[n_bins + 1]),
            "n_escaped": res.n_escaped, "n_absorbed": res.n_absorbed, "n_capped": res.n_capped,
            "sum_scat": res.sum_scat, "sum_scat2": res.sum_scat2, "sum_upar_iters": res.sum_upar_iters,
            "X0": x0, "X": x, "col": col, "nscat": rn, "status": rs}


def reweight(X0, X, col, status, *, sample, target, tau_d, n_bins, X_min, X_max):
    """Emergent spectrum reweighted from the sampled intrinsic spectrum sample = (sigma, ew, C)
    to target = (sigma, ew, C) and dust depth tau_d: sum of weights per bin / n."""
    X0 = np.ascontiguousarray(X0, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    col = np.ascontiguousarray(col, dtype=np.float64)
    st = np.ascontiguousarray(status, dtype=np.uint8)
    out = np.zeros(n_bins + 2)
    lib().orc_reweight(len(X0), _p(X0, C.c_double), _p(X, C.c_double), _p(col, C.c_double), _p(st, C.c_uint8),
                       *sample, *target, tau_d, n_bins, X_min, X_max, _p(out, C.c_double))
    return out


def dda_trace(dims, origins, dirs, max_steps):
    dims_ = np.ascontiguousarray(dims, dtype=np.int32)
    o = np.ascontiguousarray(origins, dtype=np.float64)
    d = np.ascontiguousarray(dirs, dtype=np.float32)
    n = o.shape[0]
    cells = np.full((n, max_steps), -1, dtype=np.int64)
    seg = np.zeros((n, max_steps))
    cnt = np.zeros(n, dtype=np.int32)
    lib().orc_dda_trace(_p(dims_, C.c_int32), _p(o, C.c_double), _p(d, C.c_float), n, max_steps,
                        _p(cells, C.c_int64), _p(seg, C.c_double), _p(cnt, C.c_int32))
    return cells, seg, cnt


def run_grid(fields: dict, *, cell_cm, n_photons, seed, first_id=0, phase="dipole", albedo=0.32,
             g_hg=0.73, n_bins=256, img_nx=None, X_min=-1000.0, X_max=1000.0, peel=True,
             max_scat=0, n_threads=0, raw=False, sampler="eq10"):
    nHI = np.ascontiguousarray(fields["n_HI"], dtype=np.float32)
    nz, ny, nx = nHI.shape
    arrs = [nHI] + [np.ascontiguousarray(fields[k], dtype=np.float32)
                    for k in ("T", "vx", "vy", "vz", "kd")]
    img = img_nx if img_nx else nx // 2
    run = GridRun((C.c_int32 * 3)(nx, ny, nz), PHASE[phase], cell_cm, albedo, g_hg, n_bins, img,
                  X_min, X_max, 1 if peel else 0, 0, max_scat)
    spec = np.zeros(n_bins + 2, dtype=np.uint64)
    cube = np.zeros((3, img, img, n_bins)) if peel else None
    res = Result()
    rX = np.zeros(n_photons) if raw else None
    rn = np.zeros(n_photons, np.uint64) if raw else None
    rs = np.zeros(n_photons, np.uint8) if raw else None
    rk = np.zeros((n_photons, 3)) if raw else None
    rd = np.zeros(n_photons, np.uint32) if raw else None
    with _sampler(sampler):
        lib().orc_run_grid(*[_p(a, C.c_float) for a in arrs], C.byref(run), first_id, n_photons, seed,
                           n_threads, _p(spec, C.c_uint64), _p(cube, C.c_double) if peel else None,
                           C.byref(res), _p(rX, C.c_double) if raw else None,
                           _p(rn, C.c_uint64) if raw else None, _p(rs, C.c_uint8) if raw else None,
                           _p(rk, C.c_double) if raw else None, _p(rd, C.c_uint32) if raw else None)
    out = {"counts": spec[:n_bins], "underflow": int(spec[n_bins]), "overflow": int(spec[n_bins + 1]),
           "cube": cube, "n_escaped": res.n_escaped, "n_absorbed": res.n_absorbed,
           "n_capped": res.n_capped, "sum_scat": res.sum_scat, "sum_scat2": res.sum_scat2,
           "sum_dust_scat": res.sum_dust_scat}
    if raw:
        out.update(X=rX, nscat=rn, status=rs, k=rk, ndust=rd)
    return out


def forest(n_HI, T, v_los, sel_ix, sel_iy, *, ds_cm, dv_cell, n_bins, dv_bin, n_threads=0):
    nHI = np.ascontiguousarray(n_HI, dtype=np.float32)
    Ta = np.ascontiguousarray(T, dtype=np.float32)
    va = np.ascontiguousarray(v_los, dtype=np.float32)
    nz, ny, nx = nHI.shape
    ix = np.ascontiguousarray(sel_ix, dtype=np.int32)
    iy = np.ascontiguousarray(sel_iy, dtype=np.int32)
    out = np.zeros((ix.size, n_bins))
    lib().orc_forest(_p(nHI, C.c_float), _p(Ta, C.c_float), _p(va, C.c_float), nx, ny, nz,
                     _p(ix, C.c_int32), _p(iy, C.c_int32), ix.size, ds_cm, dv_cell, n_bins, dv_bin,
                     n_threads, _p(out, C.c_double))
    return out
