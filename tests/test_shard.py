"""Sharding a batch across ranks (host side, CPU, gloo): the partition of smol_partition
and the one gather at the end. The batch's systems are independent, so each rank
integrates its own systems with no exchange; here the integrator on each rank is the
oracle (the GPU path is the same code with smol.Batch in place of the oracle call).
"""
import os
import socket

import numpy as np
import pytest

import oracle
from synth import kernel_factors, monodisperse

SPECS = [(16, 0.3, 0.01), (64, 0.7, 0.05), (33, 0.5, 0.1), (128, 0.9, 0.005), (8, 0.2, 0.02), (100, 0.4, 0.03),
         (48, 0.6, 0.01)]


@pytest.fixture(scope="module")
def smol():
    import paper_2407_16559_gb300 as m  # the partitioner is host code: no GPU needed
    return m


def test_partition_covers_and_balances(smol):
    rng = np.random.default_rng(7)
    Ms = (2 ** rng.integers(4, 17, size=300)).astype(np.int64)
    w = rng.uniform(0.5, 2.0, size=300)
    for nranks in (1, 2, 3, 8):
        rank_of, load = smol.partition(Ms, nranks, w)
        assert rank_of.min() >= 0 and rank_of.max() < nranks
        lg = np.maximum(2, np.ceil(np.log2(Ms)).astype(int))
        cost = (2.0 ** lg) * (lg + 1) * w
        assert np.allclose([cost[rank_of == r].sum() for r in range(nranks)], load)
        # LPT: the largest load exceeds the ideal share by at most the largest single cost
        assert load.max() <= cost.sum() / nranks + cost.max() + 1e-6
        again, _ = smol.partition(Ms, nranks, w)
        assert np.array_equal(rank_of, again)


def test_partition_lpt_small_case(smol):
    # costs 8*4, 8*4, 4*3, 4*3, 4*3 (M = 8, 8, 4, 4, 4): LPT gives {32, 12}, {32, 12, 12}
    rank_of, load = smol.partition([8, 8, 4, 4, 4], 2)
    assert sorted(load.tolist()) == [44.0, 56.0]
    assert rank_of.tolist() == [0, 1, 0, 1, 0]


def test_partition_rejects_bad_arguments(smol):
    with pytest.raises(smol.SmolError):
        smol.partition([8, 0], 2)
    with pytest.raises(smol.SmolError):
        smol.partition([8, 8], 0)
    with pytest.raises(smol.SmolError):
        smol.partition([8, 8], 2, weights=[1.0, -1.0])


def _integrate(spec):
    M, a, lam = spec
    U, V = kernel_factors("brownian", M, a=a)
    sysm = oracle.System(M, lam, U=U, V=V, route="direct")
    n, st, _ = oracle.integrate(sysm, monodisperse(M), 0.0, 0.3, 1e-8, oracle.Options(scheme="rkf45", tau0=1e-3))
    return n, st["accepted"], st["rejected"]


def _worker(rank, world, port, out_path, fail_rank):
    import datetime

    import torch.distributed as dist

    import paper_2407_16559_gb300 as smol
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=30))
    try:
        rank_of, _ = smol.partition([s[0] for s in SPECS], world)
        mine = smol.shard_indices(rank_of, rank)
        if rank == fail_rank:
            raise RuntimeError("injected failure on the host")
        local = [_integrate(SPECS[q]) for q in mine]
        allres = smol.gather_shards(local, rank_of, dist)
        if rank == 0:
            np.save(out_path, np.array([np.concatenate([r[0], [r[1], r[2]]]) for r in allres], dtype=object),
                    allow_pickle=True)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_batch_two_ranks_matches_one_process(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res.npy")
    mp.spawn(_worker, args=(2, _free_port(), out, -1), nprocs=2, join=True)
    got = np.load(out, allow_pickle=True)
    for q, spec in enumerate(SPECS):
        n, acc, rej = _integrate(spec)
        assert np.array_equal(got[q][:-2].astype(float), n)
        assert (int(got[q][-2]), int(got[q][-1])) == (acc, rej)


def test_sharded_batch_rank_failure_is_reported(tmp_path):
    """A rank that raises before the gather: the run ends with an error instead of
    hanging in the collective: the failing rank's own, or the other rank's gather
    seeing its peer gone (whichever process the launcher reports first)."""
    import time

    import torch.multiprocessing as mp
    t0 = time.time()
    with pytest.raises(Exception, match="injected failure|Connection closed|peer"):
        mp.spawn(_worker, args=(2, _free_port(), str(tmp_path / "x.npy"), 1), nprocs=2, join=True)
    assert time.time() - t0 < 25.0  # well inside the process group's 30 s timeout
