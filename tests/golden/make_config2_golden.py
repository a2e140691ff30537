"""Writes tests/golden/config2_full_history.json: the FP64 oracle's uncapped run of the
expanding-shell workload (THOR Sec. 3.3 shell, Sec. 3.4 transport, Sec. 4 outflow
validation geometry), the reference for the GPU test of the same workload's full photon
histories.

Workload: shell R_in = 0.9, R_out = 1, N_HI = 1e20 cm^-2, T = 1e4 K, homologous outflow
200 km/s at R_out, dust extinction 0.5 across the shell (absorbing), dipole phase function,
central source with a Gaussian line sigma = 50 km/s; 400 bins over [-1500, 1500] km/s.
Every photon runs to escape or absorption (no cap on scatterings): the ~8% of photons
trapped in the line core scatter 1e5-1e7 times, and they are the ones compared here.

The oracle runs with its default u_par sampler (Eq. 10 as printed), at a seed that no GPU
test uses.  Only oracle/ is called; nothing here comes from the CUDA path.

    python tests/golden/make_config2_golden.py [--photons 4000] [--threads 0]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402

SHELL = dict(R_in=0.9, R_out=1.0, N_HI=1e20, T=1e4, v_max=200.0, tau_dust=0.5, albedo=0.0, phase="dipole")
SOURCE = dict(line="gauss", X0=0.0, sigma=50.0)
BINS = dict(n_bins=400, X_min=-1500.0, X_max=1500.0)
SEED = 2_000_003


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--photons", type=int, default=4000)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(HERE, "config2_full_history.json"))
    a = ap.parse_args()
    geo = {k: v for k, v in SHELL.items() if k != "N_HI"}
    geo["tau0"] = SHELL["N_HI"] * oracle.line_params(SHELL["T"])["sigma0"]
    t0 = time.time()
    r = oracle.run_shell(**geo, **SOURCE, **BINS, n_photons=a.photons, seed=SEED, max_scat=0,
                         n_threads=a.threads, raw=True, sampler="eq10")
    wall = time.time() - t0
    assert r["n_capped"] == 0 and r["n_escaped"] + r["n_absorbed"] == a.photons
    out = {
        "what": "FP64 oracle, expanding shell, uncapped photon histories (THOR Sec. 3.3-3.4, Sec. 4)",
        "shell": SHELL, "source": SOURCE, "bins": BINS, "seed": SEED, "photons": a.photons,
        "upar_sampler": "eq10", "oracle_wall_s": round(wall, 1),
        "counts": [int(c) for c in r["counts"]], "underflow": r["underflow"], "overflow": r["overflow"],
        "n_escaped": int(r["n_escaped"]), "n_absorbed": int(r["n_absorbed"]),
        "sum_scat": int(r["sum_scat"]), "sum_scat2": float(r["sum_scat2"]),
        "sum_upar_iters": int(r["sum_upar_iters"]),
        "nscat": [int(v) for v in r["nscat"]], "status": [int(v) for v in r["status"]],
    }
    with open(a.out, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    ns = np.asarray(r["nscat"], dtype=np.float64)
    print(f"{a.photons} photons in {wall:.0f} s: escaped {r['n_escaped']}, absorbed {r['n_absorbed']}, "
          f"<n_scat> {ns.mean():.1f}, max {ns.max():.0f}, > 1e5: {(ns > 1e5).sum()}")


if __name__ == "__main__":
    main()
