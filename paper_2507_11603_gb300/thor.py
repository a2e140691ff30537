"""Thin ctypes binding of libthor.so (include/thor.h): argument marshalling only.

Every step of the photon loop and of the forest ray-march runs in the library's
CUDA kernels; this module converts numpy arrays / torch tensors to pointers and
back.  Loading fails loudly when the library is missing -- there is no CPU path.

Arrays: host numpy arrays are passed with THOR_MEM_HOST; torch CUDA tensors with
THOR_MEM_DEVICE (their storage is used in place, on the context's stream).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CAPACITY, ERR_TIMEOUT, ERR_DEVICE, ERR_CANCELLED, ERR_NOT_FOUND = 0, -1, -2, -3, -4, -5, -6, -7
MEM_HOST, MEM_DEVICE = 0, 1
PHASE = {"isotropic": 0, "dipole": 1, "mixed": 2}

# Every entry point declared in include/thor.h.
SYMBOLS = [
    "thor_init", "thor_destroy", "thor_last_error", "thor_ctx_set_stream", "thor_ctx_set_launch", "thor_ctx_set_tail",
    "thor_shell_create", "thor_grid_create", "thor_grid_set_scattering", "thor_geom_destroy", "thor_run",
    "thor_forest", "thor_last_elapsed_ms", "thor_server_create", "thor_server_submit", "thor_server_poll",
    "thor_server_wait", "thor_server_cancel", "thor_server_stats", "thor_server_destroy", "thor_voigt_eval",
    "thor_dda_trace", "thor_sample_upar", "thor_scatter_once", "thor_philox", "thor_line_params",
    "thor_run_shell_noalloc", "thor_noalloc_last_error", "thor_reweight", "thor_xcw_eval", "thor_ctx_set_bursts",
    "thor_issue_peak", "thor_ctx_set_grid_exec", "thor_ctx_set_tail_share",
]
PROFILE = {"homologous": 0, "power_law": 1}
SPECIES = {"HI": 0, "MgII": 1}


class ThorError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"thor error {code}: {msg}")
        self.code = code


class ShellParams(C.Structure):
    _fields_ = [("R_in", C.c_double), ("R_out", C.c_double), ("N_HI", C.c_double), ("tau0", C.c_double),
                ("T", C.c_double), ("v_max", C.c_double), ("tau_dust", C.c_double), ("albedo", C.c_double),
                ("g_hg", C.c_double), ("phase", C.c_int32), ("core_skip", C.c_int32), ("step_dx", C.c_double),
                ("profile", C.c_int32), ("species", C.c_int32), ("alpha_rho", C.c_double), ("alpha_v", C.c_double)]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("X0", C.c_double), ("sigma", C.c_double),
                ("ew", C.c_double), ("C", C.c_double)]


class OutputSpec(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("mem_kind", C.c_int32), ("X_min", C.c_double), ("X_max", C.c_double),
                ("spectrum", C.c_void_p), ("peel", C.c_int32), ("img_n", C.c_int32), ("peel_bins", C.c_int32),
                ("reserved", C.c_int32), ("peel_X_min", C.c_double), ("peel_X_max", C.c_double),
                ("cube", C.c_void_p), ("raw_X", C.c_void_p), ("raw_nscat", C.c_void_p), ("raw_status", C.c_void_p),
                ("max_scat", C.c_uint32), ("reserved2", C.c_uint32), ("raw_X0", C.c_void_p), ("raw_col", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("n_photons", C.c_uint64), ("n_escaped", C.c_uint64), ("n_absorbed", C.c_uint64),
                ("n_capped", C.c_uint64), ("n_scat", C.c_uint64), ("n_dust_scat", C.c_uint64),
                ("n_upar_iters", C.c_uint64), ("n_steps", C.c_uint64), ("n_peel_rays", C.c_uint64),
                ("n_peel_cells", C.c_uint64), ("sum_scat2", C.c_double), ("elapsed_ms", C.c_double),
                ("n_launches", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ForestSpec(C.Structure):
    _fields_ = [("ds_cm", C.c_double), ("dv_cell", C.c_double), ("n_bins", C.c_int32), ("stage_rows", C.c_int32),
                ("dv_bin", C.c_double), ("first_sightline", C.c_int64), ("n_sightlines", C.c_int64)]


class ServerConfig(C.Structure):
    _fields_ = [("max_requests", C.c_int32), ("events_per_round", C.c_int32), ("n_slots", C.c_int64),
                ("mem_budget_bytes", C.c_uint64), ("block_size", C.c_int32), ("priority", C.c_int32),
                ("presort", C.c_int32), ("reserved", C.c_int32)]


_lib = None
_lock = threading.Lock()


def load(build: bool = True) -> C.CDLL:
    """Load libthor.so (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libthor.so is missing: run paper_2507_11603_gb300._build.build()")
        L = C.CDLL(_build.LIB)
        P, vp = C.POINTER, C.c_void_p
        i32, i64, u64, dbl = C.c_int32, C.c_int64, C.c_uint64, C.c_double
        sig = {
            "thor_init": ([C.c_int, P(vp)], C.c_int),
            "thor_destroy": ([vp], None),
            "thor_last_error": ([vp], C.c_char_p),
            "thor_ctx_set_stream": ([vp, vp], C.c_int),
            "thor_ctx_set_launch": ([vp, C.c_int, C.c_int], C.c_int),
            "thor_ctx_set_tail": ([vp, C.c_int, C.c_int], C.c_int),
            "thor_ctx_set_bursts": ([vp, C.c_int, C.c_int], C.c_int),
            "thor_ctx_set_grid_exec": ([vp, C.c_int64, C.c_int64], C.c_int),
            "thor_ctx_set_tail_share": ([vp, C.c_int], C.c_int),
            "thor_shell_create": ([vp, P(ShellParams), P(vp)], C.c_int),
            "thor_grid_create": ([vp, vp, vp, vp, vp, P(i32), dbl, C.c_int, P(vp)], C.c_int),
            "thor_grid_set_scattering": ([vp, C.c_int, dbl, dbl], C.c_int),
            "thor_geom_destroy": ([vp], None),
            "thor_run": ([vp, vp, P(Source), u64, u64, u64, P(OutputSpec), P(Result)], C.c_int),
            "thor_forest": ([vp, vp, vp, vp, P(i32), C.c_int, P(ForestSpec), vp], C.c_int),
            "thor_last_elapsed_ms": ([vp], dbl),
            "thor_server_create": ([vp, P(ServerConfig), P(vp)], C.c_int),
            "thor_server_submit": ([vp, P(ShellParams), P(Source), u64, u64, P(OutputSpec), P(i64)], C.c_int),
            "thor_server_poll": ([vp, i64, P(C.c_int)], C.c_int),
            "thor_server_wait": ([vp, i64, i64, P(Result)], C.c_int),
            "thor_server_cancel": ([vp, i64], C.c_int),
            "thor_server_stats": ([vp, P(u64), P(dbl), P(u64)], C.c_int),
            "thor_server_destroy": ([vp], None),
            "thor_voigt_eval": ([vp, vp, vp, vp, i64, C.c_int, C.c_int], C.c_int),
            "thor_xcw_eval": ([vp, vp, vp, i64, C.c_int], C.c_int),
            "thor_issue_peak": ([vp, C.c_int, P(dbl)], C.c_int),
            "thor_dda_trace": ([vp, P(i32), vp, vp, i32, i32, vp, vp, vp, C.c_int], C.c_int),
            "thor_sample_upar": ([vp, C.c_float, C.c_float, u64, i64, vp, P(u64), C.c_int], C.c_int),
            "thor_scatter_once": ([vp, C.c_float, C.c_float, C.c_int, u64, i64, vp, vp, C.c_int], C.c_int),
            "thor_philox": ([vp, vp, vp, vp, i32, C.c_int], C.c_int),
            "thor_line_params": ([dbl, P(dbl), P(dbl), P(dbl)], None),
            "thor_run_shell_noalloc": ([P(ShellParams), P(Source), u64, u64, u64, i32, dbl, dbl, vp, C.c_int, vp,
                                        P(Result)], C.c_int),
            "thor_noalloc_last_error": ([], C.c_char_p),
            "thor_reweight": ([vp, i64, vp, vp, vp, vp, C.c_int, P(dbl), i32, P(dbl), i32, dbl, dbl, P(dbl)],
                              C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def line_params(T: float) -> dict:
    L = load()
    v, a, s = C.c_double(), C.c_double(), C.c_double()
    L.thor_line_params(float(T), C.byref(v), C.byref(a), C.byref(s))
    return {"vth_kms": v.value, "a": a.value, "sigma0": s.value}


def run_shell_noalloc(*, T, R_in=0.0, R_out=1.0, N_HI=0.0, tau0=0.0, v_max=0.0, tau_dust=0.0, albedo=0.0,
                      g_hg=0.73, phase="isotropic", step_dx=0.0, core_skip=False, n_photons, seed, first_id=0,
                      X0=0.0, sigma=0.0, ew=0.0, C_cont=0.0, species="HI", n_bins=200, X_min=-1000.0,
                      X_max=1000.0, spectrum=None, stream=None):
    """thor_run_shell_noalloc: the shell photon loop on the current CUDA device without any
    device allocation by the library (its scratch is a fixed static device array).  For
    callers that cannot allocate device memory at the time of the run.  `spectrum`: a host
    numpy uint64 array or a CUDA tensor of n_bins + 2 entries (allocated here as a host
    array when omitted); calls that overlap on the GPU must be serialised."""
    L = load()
    p = ShellParams(R_in, R_out, N_HI, tau0, T, v_max, tau_dust, albedo, g_hg, PHASE[phase],
                    1 if core_skip else 0, step_dx, PROFILE["homologous"], SPECIES[species])
    src = Source(0, 0, X0, sigma, ew, C_cont)
    if spectrum is None:
        spectrum = np.zeros(n_bins + 2, dtype=np.uint64)
    ptr, kind, _ = _ptr(spectrum)
    raw = getattr(stream, "cuda_stream", stream)
    res = Result()
    rc = L.thor_run_shell_noalloc(C.byref(p), C.byref(src), first_id, n_photons, seed, n_bins, X_min, X_max, ptr,
                                  kind, C.c_void_p(raw or 0), C.byref(res))
    if rc != OK:
        raise ThorError(rc, L.thor_noalloc_last_error().decode())
    return RunResult(spectrum[:n_bins], int(spectrum[n_bins]), int(spectrum[n_bins + 1]), res.as_dict())


def _ptr(x):
    """(pointer, mem_kind, keepalive) for a numpy array or a torch tensor."""
    if x is None:
        return None, MEM_HOST, None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data, MEM_HOST, x
    try:
        import torch
    except ImportError as e:  # pragma: no cover
        raise TypeError("expected a numpy array or a torch tensor") from e
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr(), (MEM_DEVICE if x.is_cuda else MEM_HOST), x
    raise TypeError("expected a numpy array or a torch tensor")


def _arr(x, name, dtype, shape=None):
    """An array argument checked before its pointer reaches the C ABI, which trusts the
    sizes it derives from dims and counts: host numpy arrays are converted to a contiguous
    array of `dtype`; tensors must already have that element type and be contiguous (a
    device tensor is never copied here); `shape`, when given, must match exactly."""
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, dtype=dtype)
    else:
        try:
            import torch
        except ImportError as e:  # pragma: no cover
            raise TypeError(f"{name}: expected a numpy array or a torch tensor") from e
        if not isinstance(x, torch.Tensor):
            raise TypeError(f"{name}: expected a numpy array or a torch tensor")
        want = {np.dtype(np.float32): torch.float32, np.dtype(np.uint8): torch.uint8}[np.dtype(dtype)]
        if x.dtype != want:
            raise TypeError(f"{name}: expected {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
    if shape is not None and tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(x.shape)}, expected {tuple(shape)}")
    return x


def _same_kind(*arrs):
    kinds = {_ptr(a)[1] for a in arrs if a is not None}
    if len(kinds) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return kinds.pop() if kinds else MEM_HOST


@dataclass
class RunResult:
    spectrum: np.ndarray
    underflow: int
    overflow: int
    stats: dict
    cube: object = None
    raw_X: object = None
    raw_nscat: object = None
    raw_status: object = None
    raw_X0: object = None
    raw_col: object = None


class Context:
    """One CUDA device (thor_init)."""

    def __init__(self, device: int = 0, block_size: int | None = None, blocks_per_sm: int = 0):
        self.L = load()
        h = C.c_void_p()
        rc = self.L.thor_init(device, C.byref(h))
        if rc != OK:
            raise ThorError(rc, self.L.thor_last_error(None).decode())
        self.h = h
        if block_size is not None:
            self._check(self.L.thor_ctx_set_launch(self.h, block_size, blocks_per_sm))

    def _check(self, rc):
        if rc != OK:
            raise ThorError(rc, self.L.thor_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.thor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self.L.thor_ctx_set_stream(self.h, C.c_void_p(raw or 0)))

    def set_launch(self, block_size: int, blocks_per_sm: int = 0):
        self._check(self.L.thor_ctx_set_launch(self.h, block_size, blocks_per_sm))

    def set_bursts(self, pipe_lanes: int = 32, burst_lanes: int = 1):
        """thor_ctx_set_bursts: pipelined events in warps with at most pipe_lanes live packets,
        core bursts in warps with at most burst_lanes (0 = never); results do not depend on
        them."""
        self._check(self.L.thor_ctx_set_bursts(self.h, pipe_lanes, burst_lanes))

    def set_grid_exec(self, slots: int = 0, handoff: int | None = None):
        """thor_ctx_set_grid_exec: event-based grid loop with `slots` packets in flight
        (0 = the one-kernel loop), handing the last `handoff` (default slots // 8) to the
        one-kernel loop; results do not depend on it."""
        if handoff is None:
            handoff = slots // 8
        self._check(self.L.thor_ctx_set_grid_exec(self.h, int(slots), int(handoff)))

    def set_tail_share(self, share: bool = True):
        """thor_ctx_set_tail_share: work sharing in the tail of a one-launch shell run (on by
        default); results do not depend on it."""
        self._check(self.L.thor_ctx_set_tail_share(self.h, 1 if share else 0))

    def set_tail(self, spill_below: int = 0, max_phases: int = 24):
        """thor_ctx_set_tail: tail compaction of the shell photon loop (0 = off, the library's
        default); results do not depend on it."""
        self._check(self.L.thor_ctx_set_tail(self.h, spill_below, max_phases))

    # -------------------------------------------------------------- geometries
    def shell(self, *, T, R_in=0.0, R_out=1.0, N_HI=0.0, tau0=0.0, v_max=0.0, tau_dust=0.0, albedo=0.0, g_hg=0.73,
              phase="isotropic", step_dx=0.0, core_skip=False, profile="homologous", alpha_rho=0.0, alpha_v=1.0,
              species="HI"):
        """thor_shell_create.  profile "power_law": the Sec. 5.1 geometry, v_max = distance-averaged
        speed; species "MgII" (power law): the doublet, N_HI = the Mg II column."""
        p = ShellParams(R_in, R_out, N_HI, tau0, T, v_max, tau_dust, albedo, g_hg, PHASE[phase],
                        1 if core_skip else 0, step_dx, PROFILE[profile], SPECIES[species], alpha_rho, alpha_v)
        g = C.c_void_p()
        self._check(self.L.thor_shell_create(self.h, C.byref(p), C.byref(g)))
        return Geometry(self, g, "shell", params=p)

    def grid(self, n_HI, T, v, dust, cell_cm, phase="dipole", albedo=0.32, g_hg=0.73):
        """Fields of shape (nz, ny, nx); v of shape (3, nz, ny, nx) (vx, vy, vz)."""
        n_HI = _arr(n_HI, "n_HI", np.float32)
        if len(n_HI.shape) != 3:
            raise ValueError("n_HI must have shape (nz, ny, nx)")
        shape = tuple(n_HI.shape)
        T = _arr(T, "T", np.float32, shape)
        v = _arr(v, "v", np.float32, (3,) + shape)
        dust = None if dust is None else _arr(dust, "dust", np.float32, shape)
        kind = _same_kind(n_HI, T, v, dust)
        nz, ny, nx = shape
        dims = (C.c_int32 * 3)(nx, ny, nz)
        g = C.c_void_p()
        self._check(self.L.thor_grid_create(self.h, _ptr(n_HI)[0], _ptr(T)[0], _ptr(v)[0], _ptr(dust)[0], dims,
                                            float(cell_cm), kind, C.byref(g)))
        geo = Geometry(self, g, "grid", dims=(nx, ny, nz))
        self._check(self.L.thor_grid_set_scattering(g, PHASE[phase], float(albedo), float(g_hg)))
        return geo

    # -------------------------------------------------------------- runs
    def run(self, geom, *, n_photons, seed, first_id=0, X0=0.0, sigma=0.0, ew=0.0, C_cont=0.0, n_bins=200,
            X_min=-1000.0, X_max=1000.0, peel=False, img_n=128, peel_bins=256, peel_X_min=-1000.0,
            peel_X_max=1000.0, raw=False, raw_sweep=False, max_scat=0, device_out=False):
        """thor_run: photons first_id .. first_id + n_photons - 1 of stream `seed`.  raw_sweep
        (power-law shells) also returns the emitted X0 and the HI column of every photon."""
        src = Source(1 if geom.kind == "grid" else 0, 0, X0, sigma, ew, C_cont)
        torch = None
        if device_out:
            import torch
            spec_arr = torch.zeros(n_bins + 2, dtype=torch.int64, device="cuda")
            mk = MEM_DEVICE
        else:
            spec_arr = np.zeros(n_bins + 2, dtype=np.uint64)
            mk = MEM_HOST
        cube = rX = rn = rs = None
        if peel:
            shape = (3, img_n, img_n, peel_bins)
            cube = torch.zeros(shape, dtype=torch.float32, device="cuda") if device_out else np.zeros(shape, np.float32)
        if raw:
            if device_out:
                rX = torch.zeros(n_photons, dtype=torch.float32, device="cuda")
                rn = torch.zeros(n_photons, dtype=torch.int32, device="cuda")
                rs = torch.zeros(n_photons, dtype=torch.uint8, device="cuda")
            else:
                rX, rn, rs = np.zeros(n_photons, np.float32), np.zeros(n_photons, np.uint32), np.zeros(n_photons, np.uint8)
        r0 = rc = None
        if raw_sweep:
            if device_out:
                r0 = torch.zeros(n_photons, dtype=torch.float32, device="cuda")
                rc = torch.zeros(n_photons, dtype=torch.float32, device="cuda")
            else:
                r0, rc = np.zeros(n_photons, np.float32), np.zeros(n_photons, np.float32)
        spec = OutputSpec(n_bins, mk, X_min, X_max, _ptr(spec_arr)[0], 1 if peel else 0, img_n, peel_bins, 0,
                          peel_X_min, peel_X_max, _ptr(cube)[0] if peel else None,
                          _ptr(rX)[0] if raw else None, _ptr(rn)[0] if raw else None, _ptr(rs)[0] if raw else None,
                          max_scat, 0, _ptr(r0)[0] if raw_sweep else None, _ptr(rc)[0] if raw_sweep else None)
        res = Result()
        self._check(self.L.thor_run(self.h, geom.h, C.byref(src), first_id, n_photons, seed, C.byref(spec),
                                    C.byref(res)))
        counts = spec_arr if not device_out else spec_arr
        return RunResult(counts[:n_bins], int(counts[n_bins]), int(counts[n_bins + 1]), res.as_dict(), cube, rX, rn, rs,
                         r0, rc)

    def reweight(self, X0, X, col, status, *, sample, targets, n_bins, X_min, X_max):
        """thor_reweight: spectra of the escaped photons for each target (sigma, ew, C, tau_d),
        reweighted from the sampled intrinsic spectrum sample = (sigma, ew, C); shape
        (n_targets, n_bins + 2), sum of weights per bin / n."""
        X0 = _arr(X0, "X0", np.float32)
        if len(X0.shape) != 1:
            raise ValueError("X0 must be one-dimensional")
        n = int(X0.shape[0])
        X = _arr(X, "X", np.float32, (n,))
        col = _arr(col, "col", np.float32, (n,))
        status = _arr(status, "status", np.uint8, (n,))
        kind = _same_kind(X0, X, col, status)
        smp = (C.c_double * 3)(*[float(v) for v in sample])
        tg = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(-1, 4))
        out = np.zeros((tg.shape[0], n_bins + 2))
        self._check(self.L.thor_reweight(self.h, n, _ptr(X0)[0], _ptr(X)[0], _ptr(col)[0], _ptr(status)[0], kind, smp,
                                         tg.shape[0], tg.ctypes.data_as(C.POINTER(C.c_double)), n_bins, float(X_min),
                                         float(X_max), out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def forest(self, n_HI, T, v_los, *, ds_cm, dv_cell, n_bins, dv_bin, first=0, count=None, out=None,
               stage_rows=0):
        """thor_forest; stage_rows: rows of sightlines per staged chunk for host arrays (0 = automatic)."""
        n_HI = _arr(n_HI, "n_HI", np.float32)
        if len(n_HI.shape) != 3:
            raise ValueError("n_HI must have shape (nz, ny, nx)")
        shape = tuple(n_HI.shape)
        T = _arr(T, "T", np.float32, shape)
        v_los = _arr(v_los, "v_los", np.float32, shape)
        kind = _same_kind(n_HI, T, v_los)
        nz, ny, nx = shape
        count = nx * ny - first if count is None else count
        if out is None:
            if kind == MEM_DEVICE:
                import torch
                out = torch.empty((count, n_bins), dtype=torch.float32, device=n_HI.device)
            else:
                out = np.zeros((count, n_bins), np.float32)
        elif isinstance(out, np.ndarray) and (out.dtype != np.float32 or not out.flags["C_CONTIGUOUS"]):
            raise TypeError("out must be a C-contiguous float32 array")  # written in place: no conversion
        else:
            out = _arr(out, "out", np.float32, (count, n_bins))
        if _same_kind(out) != kind:
            raise ValueError("out must live where the fields live (host or device)")
        if tuple(out.shape) != (count, n_bins):
            raise ValueError(f"out: shape {tuple(out.shape)}, expected {(count, n_bins)}")
        dims = (C.c_int32 * 3)(nx, ny, nz)
        sp = ForestSpec(ds_cm, dv_cell, n_bins, int(stage_rows), dv_bin, first, count)
        self._check(self.L.thor_forest(self.h, _ptr(n_HI)[0], _ptr(T)[0], _ptr(v_los)[0], dims, kind, C.byref(sp),
                                       _ptr(out)[0]))
        return out

    def last_elapsed_ms(self) -> float:
        return self.L.thor_last_elapsed_ms(self.h)

    # -------------------------------------------------------------- diagnostics
    def voigt(self, a, x, precise=True):
        a = np.ascontiguousarray(a, np.float32)
        x = np.ascontiguousarray(x, np.float32)
        a, x = np.broadcast_arrays(a, x)
        a, x = np.ascontiguousarray(a), np.ascontiguousarray(x)
        H = np.zeros(x.shape, np.float32)
        self._check(self.L.thor_voigt_eval(self.h, a.ctypes.data, x.ctypes.data, H.ctypes.data, x.size,
                                           1 if precise else 0, MEM_HOST))
        return H

    def xcw(self, a):
        """Core-to-wing transition x_cw(a) (App. A.2) as the device computes it (B25, fast log)."""
        a = np.ascontiguousarray(a, np.float32)
        out = np.zeros(a.shape, np.float32)
        self._check(self.L.thor_xcw_eval(self.h, a.ctypes.data, out.ctypes.data, a.size, MEM_HOST))
        return out

    def issue_peak(self, kind: str = "fma") -> float:
        """thor_issue_peak: measured warp instructions per second of FP32 FMA ("fma") or MUFU
        ex2 ("mufu") over the whole device."""
        v = C.c_double()
        self._check(self.L.thor_issue_peak(self.h, {"fma": 0, "mufu": 1}[kind], C.byref(v)))
        return v.value

    def dda(self, dims, origins, dirs, max_steps):
        o = np.ascontiguousarray(origins, np.float64)
        d = np.ascontiguousarray(dirs, np.float32)
        n = o.shape[0]
        if o.shape != (n, 3) or d.shape != (n, 3):
            raise ValueError("origins and dirs must both have shape (n, 3)")
        cells = np.full((n, max_steps), -1, np.int64)
        seg = np.zeros((n, max_steps))
        cnt = np.zeros(n, np.int32)
        dm = (C.c_int32 * 3)(*[int(v) for v in dims])
        self._check(self.L.thor_dda_trace(self.h, dm, o.ctypes.data, d.ctypes.data, n, max_steps, cells.ctypes.data,
                                          seg.ctypes.data, cnt.ctypes.data, MEM_HOST))
        return cells, seg, cnt

    def sample_upar(self, x, a, n, seed=0):
        out = np.zeros(n, np.float32)
        it = C.c_uint64()
        self._check(self.L.thor_sample_upar(self.h, float(x), float(a), seed, n, out.ctypes.data, C.byref(it), MEM_HOST))
        return out, it.value

    def scatter_once(self, x, a, phase, n, seed=0):
        xo = np.zeros(n, np.float32)
        mu = np.zeros(n, np.float32)
        self._check(self.L.thor_scatter_once(self.h, float(x), float(a), int(phase), seed, n, xo.ctypes.data,
                                             mu.ctypes.data, MEM_HOST))
        return xo, mu

    def philox(self, ctr, key):
        ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
        key = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
        out = np.zeros_like(ctr)
        self._check(self.L.thor_philox(self.h, ctr.ctypes.data, key.ctypes.data, out.ctypes.data, ctr.shape[0], MEM_HOST))
        return out

    def server(self, *, max_requests=256, events_per_round=256, n_slots=0, mem_budget_bytes=0, block_size=0,
               priority=True, presort=False):
        """thor_server_create; priority: age priority (the oldest requests' packets one per warp);
        presort: frequency pre-sorting of the packets in flight between rounds."""
        return Server(self, ServerConfig(max_requests, events_per_round, n_slots, mem_budget_bytes, block_size,
                                         0 if priority else -1, 1 if presort else 0, 0))


class Geometry:
    def __init__(self, ctx, h, kind, dims=None, params=None):
        self.ctx, self.h, self.kind, self.dims, self.params = ctx, h, kind, dims, params

    def close(self):
        if self.h:
            self.ctx.L.thor_geom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """thor_server_*: continuous batching of shell-model requests."""

    def __init__(self, ctx: Context, cfg: ServerConfig):
        self.ctx = ctx
        h = C.c_void_p()
        ctx._check(ctx.L.thor_server_create(ctx.h, C.byref(cfg), C.byref(h)))
        self.h = h
        self._bufs = {}

    def submit(self, *, T, R_in=0.9, R_out=1.0, N_HI=0.0, tau0=0.0, v_max=0.0, tau_dust=0.0, albedo=0.0,
               g_hg=0.73, phase="dipole", step_dx=0.0, n_photons, seed, X0=0.0, sigma=0.0, ew=0.0, C_cont=0.0,
               n_bins=400, X_min=-1500.0, X_max=1500.0, max_scat=0, core_skip=False, profile="homologous",
               alpha_rho=0.0, alpha_v=1.0):
        p = ShellParams(R_in, R_out, N_HI, tau0, T, v_max, tau_dust, albedo, g_hg, PHASE[phase],
                        1 if core_skip else 0, step_dx, PROFILE[profile], 0, alpha_rho, alpha_v)
        src = Source(0, 0, X0, sigma, ew, C_cont)
        buf = np.zeros(n_bins + 2, np.uint64)
        spec = OutputSpec(n_bins, MEM_HOST, X_min, X_max, buf.ctypes.data, 0, 0, 0, 0, 0.0, 0.0, None, None, None,
                          None, max_scat, 0, None, None)
        t = C.c_int64()
        self.ctx._check(self.ctx.L.thor_server_submit(self.h, C.byref(p), C.byref(src), n_photons, seed, C.byref(spec),
                                                      C.byref(t)))
        self._bufs[t.value] = (buf, n_bins)
        return t.value

    def poll(self, ticket) -> bool:
        d = C.c_int()
        self.ctx._check(self.ctx.L.thor_server_poll(self.h, ticket, C.byref(d)))
        return bool(d.value)

    def wait(self, ticket, timeout_ms=-1):
        r = Result()
        self.ctx._check(self.ctx.L.thor_server_wait(self.h, ticket, int(timeout_ms), C.byref(r)))
        buf, nb = self._bufs.pop(ticket)
        return RunResult(buf[:nb].copy(), int(buf[nb]), int(buf[nb + 1]), r.as_dict())

    def cancel(self, ticket):
        self.ctx._check(self.ctx.L.thor_server_cancel(self.h, ticket))

    def stats(self):
        r, m, a = C.c_uint64(), C.c_double(), C.c_uint64()
        self.ctx._check(self.ctx.L.thor_server_stats(self.h, C.byref(r), C.byref(m), C.byref(a)))
        return {"rounds": r.value, "mean_resident": m.value, "admitted": a.value}

    def close(self):
        if self.h:
            self.ctx.L.thor_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
