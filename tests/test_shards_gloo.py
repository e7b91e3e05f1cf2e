"""Multi-process sharding of the walkers, on CPU with the gloo backend.

Walkers are independent chains (Section 4.1) and every random number is a
function of (seed, iteration, global walker index), so N ranks that each run
walkers [rank z, (rank + 1) z) with walker0 = rank z reproduce, together, the
single run of N z walkers; the benchmark's per-rank timing is combined with a
MAX all-reduce.  Both rules are exercised here with two gloo ranks driving the
oracle (the GPU path uses the same walker0 rule, tested on one GPU in
test_gpu_scale).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2104_07097_gb300 import workloads as wl

Z, STEPS, SEED = 24, 15, 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = wl.random_polytope(8, 40, seed=3)
        X0 = np.tile(p.x0, (Z, 1))
        res = oracle.mhar_run(p.A, p.b, X0, STEPS, thin=5, seed=SEED, walker0=rank * Z)
        mine = torch.from_numpy(res["samples"].copy())
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        # per-rank "time", combined the way the benchmark combines step times
        t = torch.tensor([float(rank + 1)])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            np.save(os.path.join(outdir, "gathered.npy"), torch.cat(parts, dim=1).numpy())
            np.save(os.path.join(outdir, "tmax.npy"), t.numpy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_unsharded_run(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    got = np.load(tmp_path / "gathered.npy")
    p = wl.random_polytope(8, 40, seed=3)
    ref = oracle.mhar_run(p.A, p.b, np.tile(p.x0, (world * Z, 1)), STEPS, thin=5, seed=SEED)
    np.testing.assert_array_equal(got, ref["samples"])
    assert float(np.load(tmp_path / "tmax.npy")[0]) == pytest.approx(2.0)


def _moments(snaps, shift):
    """s1, s2 and count of the points of every snapshot about `shift`."""
    pts = np.vstack(snaps) - shift
    return pts.sum(axis=0), pts.T @ pts, pts.shape[0]


def _fit_rank_main(rank, world, port, outdir):
    # Each rank warms up its own walkers, takes the moments of its snapshot
    # points about the common shift x0, and the SUM all-reduce pools them:
    # the pooled fit is the fit of all the ranks' points (the rule behind
    # mhar_fit_moments / mhar_fit_from_moments).
    import oracle.precond as opc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = wl.random_polytope(8, 40, seed=3)
        res = oracle.mhar_run(p.A, p.b, np.tile(p.x0, (Z, 1)), STEPS, thin=1, seed=SEED,
                              walker0=rank * Z)
        snaps = [res["samples"][t - 1] for t in (9, 12, 15)]
        s1, s2, cnt = _moments(snaps, p.x0)
        buf = torch.from_numpy(np.concatenate([s1, s2.ravel(), [float(cnt)]]))
        dist.all_reduce(buf, op=dist.ReduceOp.SUM)
        v = buf.numpy()
        n = p.n
        s1, s2, cnt = v[:n], v[n:n + n * n].reshape(n, n), v[-1]
        Sigma = (s2 - np.outer(s1, s1) / cnt) / (cnt - 1)
        delta, U = opc.fit(Sigma, 3, 4, seed=SEED)
        if rank == 0:
            np.save(os.path.join(outdir, "sigma.npy"), Sigma)
            np.save(os.path.join(outdir, "delta.npy"), delta)
    finally:
        dist.destroy_process_group()


def test_pooled_preconditioner_fit_over_gloo_ranks(tmp_path):
    import oracle.precond as opc
    world = 2
    mp.start_processes(_fit_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    p = wl.random_polytope(8, 40, seed=3)
    res = oracle.mhar_run(p.A, p.b, np.tile(p.x0, (world * Z, 1)), STEPS, thin=1, seed=SEED)
    snaps = [res["samples"][t - 1] for t in (9, 12, 15)]
    want_sigma = opc.covariance(snaps)
    got_sigma = np.load(tmp_path / "sigma.npy")
    np.testing.assert_allclose(got_sigma, want_sigma, rtol=1e-10,
                               atol=1e-12 * np.abs(want_sigma).max())
    delta, _ = opc.fit(want_sigma, 3, 4, seed=SEED)
    np.testing.assert_allclose(np.load(tmp_path / "delta.npy"), delta, rtol=1e-8)
