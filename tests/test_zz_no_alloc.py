"""thor_run_shell_noalloc, the entry point for callers that cannot allocate device memory
when they need a run (an external pool with nothing to spare, a used-up GPU quota, a
host callback where cudaMalloc is not allowed).  It must give the same result as the
allocating thor_run on the same arguments, twice in a row (its static scratch keeps the
previous call's contents, which the call has to clear).  Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_thor_run_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11603_gb300 import thor
    geo = dict(R_in=0.9, N_HI=1e19, T=1e4, v_max=150.0, tau_dust=0.4, phase="dipole")
    run = dict(n_photons=20000, seed=31, sigma=50.0, n_bins=300, X_min=-1500.0, X_max=1500.0)
    # first call on this device: set-up happens here, outside any stream capture
    a = thor.run_shell_noalloc(**geo, **run)
    b = thor.run_shell_noalloc(**geo, **run)
    dev = torch.zeros(run["n_bins"] + 2, dtype=torch.int64, device="cuda")
    c = thor.run_shell_noalloc(**geo, **run, spectrum=dev)
    ctx = thor.Context(0)
    ref = ctx.run(ctx.shell(**geo), n_photons=run["n_photons"], seed=run["seed"], sigma=run["sigma"],
                  n_bins=run["n_bins"], X_min=run["X_min"], X_max=run["X_max"])
    ctx.close()
    # integer tallies: the tolerance of the photon-loop parity tests for counts is exact
    for r in (a, b):
        assert np.array_equal(r.spectrum, ref.spectrum)
        assert (r.underflow, r.overflow) == (ref.underflow, ref.overflow)
        for k in ("n_escaped", "n_absorbed", "n_capped", "n_scat", "n_dust_scat"):
            assert r.stats[k] == ref.stats[k], k
    assert np.array_equal(c.spectrum.cpu().numpy().astype(np.uint64), ref.spectrum)
    assert c.stats["n_scat"] == ref.stats["n_scat"]


def test_noalloc_bins_like_thor_run():
    """Binnings whose scale rounds differently in FP32 depending on how it is formed (300 bins
    over [-40, 40] km/s: 3.7499998 or 3.75 per km/s): photons at bin edges land in the same
    bins as through thor_run, twice in a row."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11603_gb300 import thor
    geo = dict(tau0=1e4, T=1e4, phase="isotropic")
    ctx = thor.Context(0)
    g = ctx.shell(**geo)
    for nb, lo, hi in ((300, -40.0, 40.0), (1000, -30.0, 30.0)):
        run = dict(n_photons=20000, seed=5, n_bins=nb, X_min=lo, X_max=hi)
        ref = ctx.run(g, **run)
        for _ in range(2):
            r = thor.run_shell_noalloc(**geo, **run)
            assert np.array_equal(r.spectrum, ref.spectrum), (nb, lo, hi)
            assert (r.underflow, r.overflow) == (ref.underflow, ref.overflow)
    ctx.close()


def test_noalloc_rejects_oversized_host_spectrum():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11603_gb300 import thor
    with pytest.raises(thor.ThorError) as e:
        thor.run_shell_noalloc(T=1e4, tau0=10.0, n_photons=10, seed=1, n_bins=4097)
    assert e.value.code == thor.ERR_CAPACITY
