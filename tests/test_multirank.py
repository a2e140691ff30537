"""N > 1 path on CPU: world-size-2 gloo ranks shard photon ids and merge integer
spectra; the merged result equals a single-rank run exactly (the per-rank compute
here is the oracle, which keys every photon's stream by its global id just as the
device path does)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2507_11603_gb300 import sharding

KW = dict(tau0=3e3, T=1e4, R_in=0.5, v_max=50.0, tau_dust=0.3, phase="dipole", line="gauss", sigma=30.0,
          seed=17, n_bins=48, X_min=-400.0, X_max=400.0, n_threads=2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_per_rank, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, n = sharding.photon_range(rank, world, n_per_rank)
    r = oracle.run_shell(n_photons=n, first_id=first, **KW)
    counts = torch.as_tensor(np.concatenate([r["counts"].astype(np.int64),
                                             [r["n_escaped"], r["n_absorbed"], r["sum_scat"]]]))
    merged = sharding.merge_counts(counts)
    if rank == 0:
        q.put(merged.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_rank(orc):
    world, n_per_rank = 2, 600
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_per_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    r = orc.run_shell(n_photons=world * n_per_rank, first_id=0, **KW)
    single = np.concatenate([r["counts"].astype(np.int64), [r["n_escaped"], r["n_absorbed"], r["sum_scat"]]])
    assert np.array_equal(merged, single)


def test_ranges_partition_ids():
    for world in (1, 2, 3, 8):
        got = []
        for rank in range(world):
            f, n = sharding.split_range(rank, world, 1001)
            got.extend(range(f, f + n))
        assert got == list(range(1001))
        f0, n0 = sharding.photon_range(world - 1, world, 10, base=5)
        assert f0 == 5 + (world - 1) * 10 and n0 == 10
    with pytest.raises(ValueError):
        sharding.photon_range(2, 2, 10)


PL = dict(dv_ratio=5.0, N_HI=10 ** 17.4, T=1e4, v_avg=120.0, alpha_rho=-1.0, alpha_v=0.5, sigma=800.0, ew=740.0,
          C_cont=2500.0, seed=23, n_bins=30, X_min=-2500.0, X_max=2500.0, n_threads=2)
SAMPLE, TARGET = (800.0, 740.0, 2500.0), (300.0, 24661.0, 2500.0)


def _sweep_worker(rank, world, port, n_per_rank, q):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, n = sharding.photon_range(rank, world, n_per_rank)
    r = oracle.run_plshell(n_photons=n, first_id=first, **PL)
    h = oracle.reweight(r["X0"], r["X"], r["col"], r["status"], sample=SAMPLE, target=TARGET, tau_d=0.4,
                        n_bins=30, X_min=-2500.0, X_max=2500.0)
    merged = sharding.merge_weights(h, n)
    if rank == 0:
        q.put(merged.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_sweep_reweighting_over_two_gloo_ranks(orc):
    """Sharded shell-model sweep: ranks run their photon ids of a power-law shell, reweight
    their own escaped photons and merge the weighted spectra; the result equals a
    single-rank run reweighted at once (up to the order of the FP64 sums)."""
    world, n_per_rank = 2, 300
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sweep_worker, args=(r, world, port, n_per_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    r = orc.run_plshell(n_photons=world * n_per_rank, first_id=0, **PL)
    single = orc.reweight(r["X0"], r["X"], r["col"], r["status"], sample=SAMPLE, target=TARGET, tau_d=0.4,
                          n_bins=30, X_min=-2500.0, X_max=2500.0)
    assert np.allclose(merged, single, rtol=1e-12, atol=1e-15)
