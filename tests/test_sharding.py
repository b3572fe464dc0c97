"""Multi-rank logic of the realization sharding, as gloo processes on CPU.

The FP64 oracle stands in for the kernels: each rank simulates its own
pair-aligned range of realizations, the pieces are gathered, and the result
must equal one unsharded run.  The timing reduction (slowest rank) is checked
the same way.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2109_11044_gb300 import shard


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("R_total", [0, 1, 2, 5, 10, 100, 101])
def test_pair_aligned_shard_partitions_the_range(world, R_total):
    covered = []
    for rank in range(world):
        r0, cnt = shard.pair_aligned_shard(R_total, rank, world)
        assert r0 % 2 == 0 and cnt >= 0
        covered.extend(range(r0, r0 + cnt))
    assert covered == list(range(R_total))
    loads = [shard.pair_aligned_shard(R_total, k, world)[1] for k in range(world)]
    assert max(loads) - min(loads) <= 2 + R_total % 2   # whole pairs; an odd total leaves one half pair


def test_weak_offsets_are_even_and_disjoint():
    for R in (1, 2, 7, 100):
        offs = [shard.weak_offset(R, k) for k in range(5)]
        assert all(o % 2 == 0 for o in offs)
        assert all(b - a >= R for a, b in zip(offs, offs[1:]))
    with pytest.raises(ValueError):
        shard.pair_aligned_shard(4, 2, 2)


def _problem():
    m = 12
    prob = oracle.Problem(m, 0.0, 0.0, 1.0 / (m - 1), 1.0, 0.25, 0.5, 0.08)
    rng = np.random.default_rng(11)
    sites = rng.uniform(0.0, 1.0, (9, 2))
    oracle.setup_local(prob, sites, rng.standard_normal(9), 2)
    return prob


R_TOTAL, SEED = 7, 77


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r0, cnt = shard.pair_aligned_shard(R_TOTAL, rank, world)
        piece = oracle.condsim(_problem(), SEED, r0, cnt) if cnt else np.zeros((0, 12, 12))
        full = shard.gather_realizations(torch.from_numpy(np.ascontiguousarray(piece)), R_TOTAL)
        slowest = shard.max_over_ranks(1.5 + rank)
        # ensemble moments: each rank's per-node sums (what ce_ensemble_moments leaves on its
        # GPU), added over ranks by the one exchange the sharded ensemble has
        sums = (torch.from_numpy(piece.sum(axis=0)), torch.from_numpy((piece * piece).sum(axis=0)))
        count = shard.allreduce_moments(sums, cnt)
        if rank == 0:
            np.save(os.path.join(outdir, "gathered.npy"), full.numpy())
            np.save(os.path.join(outdir, "slowest.npy"), np.array([slowest]))
            np.save(os.path.join(outdir, "moments.npy"), np.stack([sums[0].numpy(), sums[1].numpy()]))
            np.save(os.path.join(outdir, "count.npy"), np.array([count]))
    finally:
        torch.distributed.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reassemble_the_unsharded_ensemble(world, tmp_path):
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    gathered = np.load(tmp_path / "gathered.npy")
    whole = oracle.condsim(_problem(), SEED, 0, R_TOTAL)
    assert gathered.shape == whole.shape
    assert np.allclose(gathered, whole, rtol=0, atol=1e-12)
    assert float(np.load(tmp_path / "slowest.npy")[0]) == 1.5 + (world - 1)
    mom = np.load(tmp_path / "moments.npy")
    assert int(np.load(tmp_path / "count.npy")[0]) == R_TOTAL
    assert np.allclose(mom[0], whole.sum(axis=0), rtol=1e-12, atol=1e-12)
    assert np.allclose(mom[1], (whole * whole).sum(axis=0), rtol=1e-12, atol=1e-12)


def test_single_process_helpers_are_identities():
    x = torch.arange(6.0).reshape(3, 2)
    assert shard.max_over_ranks(3.25) == 3.25
    assert torch.equal(shard.gather_realizations(x, 3), x)
    assert shard.allreduce_moments((x, x * x), 3) == 3
