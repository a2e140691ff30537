"""The C-ABI library builds, loads and exports every symbol include/thor.h declares;
the product path never reaches the oracle.  CPU only (no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "thor.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(thor_\w+)\s*\(", src)))


def test_header_declarations_match_binding():
    from paper_2507_11603_gb300 import thor
    assert _declared() == sorted(thor.SYMBOLS)


def test_library_builds_and_exports_symbols():
    import ctypes
    from paper_2507_11603_gb300 import _build
    lib = _build.build()
    L = ctypes.CDLL(lib)
    for name in _declared():
        assert hasattr(L, name), name


def test_library_is_sm103a_only():
    from paper_2507_11603_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_init_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2507_11603_gb300 import thor
    with pytest.raises(thor.ThorError) as e:
        thor.Context(0)
    assert e.value.code == thor.ERR_DEVICE


def test_shell_parameters_checked_before_the_device():
    """Non-finite or out-of-range shell parameters are rejected with INVALID_ARG before any
    CUDA call (so this runs without a GPU); valid ones get as far as the device.  The
    allocation-free entry point runs the checks of thor_shell_create and thor_run: negative
    or non-finite continuum and equivalent width, a continuum on a homologous shell, and the
    Mg II doublet on a homologous shell are all refused."""
    import torch
    from paper_2507_11603_gb300 import thor
    base = dict(T=1e4, tau0=1e4, n_photons=10, seed=1, n_bins=8)
    for bad in (dict(T=float("inf")), dict(T=float("nan")), dict(T=0.0), dict(tau0=float("inf")),
                dict(v_max=float("nan")), dict(tau_dust=float("inf")), dict(R_out=float("inf")),
                dict(tau0=1e300), dict(step_dx=float("nan")), dict(X0=float("nan")), dict(sigma=float("inf")),
                dict(C_cont=-1.0), dict(C_cont=float("nan")), dict(ew=-1.0), dict(ew=float("inf")),
                dict(C_cont=100.0, sigma=50.0), dict(species="MgII")):
        with pytest.raises(thor.ThorError) as e:
            thor.run_shell_noalloc(**{**base, **bad})
        assert e.value.code == thor.ERR_INVALID_ARG, bad
    if not torch.cuda.is_available():
        with pytest.raises(thor.ThorError) as e:
            thor.run_shell_noalloc(**base)
        assert e.value.code == thor.ERR_DEVICE


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2507_11603_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "thor_oracle" not in txt and "liboracle" not in txt, f
    # and the oracle never reaches the product
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".cpp")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2507_11603_gb300" not in txt and "thor_device" not in txt, f


def test_line_params_host_function():
    from paper_2507_11603_gb300 import thor
    p = thor.line_params(1e4)
    assert abs(p["vth_kms"] - 12.845) < 1e-3
    assert abs(p["a"] - 4.718e-4) < 1e-6


def test_binding_checks_arrays_before_the_call():
    """The C ABI trusts the sizes it derives from dims and counts, so the binding checks
    element types and shapes first: a short or half-precision field would otherwise be
    read past its end on the device.  Host arrays of another float type are converted."""
    import numpy as np
    import torch
    from paper_2507_11603_gb300 import thor
    C = thor.Context  # unbound: every check below raises before the library is touched
    f32 = np.zeros((4, 3, 2), np.float32)
    v = np.zeros((3, 4, 3, 2), np.float32)
    with pytest.raises(ValueError):
        C.grid(object(), f32, f32, f32, None, 1.0)  # v without its leading axis of 3
    with pytest.raises(ValueError):
        C.grid(object(), f32, f32[:3], v, None, 1.0)
    with pytest.raises(ValueError):
        C.grid(object(), f32, f32, v, np.zeros(5, np.float32), 1.0)
    with pytest.raises(TypeError):
        C.grid(object(), torch.zeros((4, 3, 2), dtype=torch.float16), f32, v, None, 1.0)
    with pytest.raises(ValueError):
        C.forest(object(), f32, f32, np.zeros((4, 3), np.float32), ds_cm=1.0, dv_cell=1.0, n_bins=4, dv_bin=1.0)
    with pytest.raises(TypeError):
        C.forest(object(), f32, f32, f32, ds_cm=1.0, dv_cell=1.0, n_bins=4, dv_bin=1.0,
                 out=np.zeros((6, 4), np.float64))
    with pytest.raises(ValueError):
        C.forest(object(), f32, f32, f32, ds_cm=1.0, dv_cell=1.0, n_bins=4, dv_bin=1.0,
                 out=np.zeros((5, 4), np.float32))
    x = np.zeros(10, np.float32)
    with pytest.raises(ValueError):
        C.reweight(object(), x, x[:9], x, np.zeros(10, np.uint8), sample=(1, 1, 1), targets=[1, 1, 1, 0],
                   n_bins=4, X_min=-1, X_max=1)
    with pytest.raises(TypeError):
        C.reweight(object(), x, x, x, torch.zeros(10, dtype=torch.int32), sample=(1, 1, 1), targets=[1, 1, 1, 0],
                   n_bins=4, X_min=-1, X_max=1)
    with pytest.raises(ValueError):
        C.dda(object(), (2, 2, 2), np.zeros((5, 3)), np.zeros((4, 3), np.float32), 8)
    # a float64 host field is converted, not rejected
    assert thor._arr(np.zeros((2, 2)), "x", np.float32).dtype == np.float32
