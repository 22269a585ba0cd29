"""Column-sharded sequence over CPU ranks (gloo, world size 2 and 3): slab
bounds, the padded all-gather and the column order.  Each rank computes its
slab with the oracle on the slab of Y it owns; the gathered sequence must
equal the oracle's sequence of the whole block."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_0704_2351_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    A = synth.planted_sparse(120, 100, 80, row_len=5, seed=4)
    return A, 65521, 3, 7, 9, 30  # A, p, m, n, seed, L


def _oracle_slab(c0, w):
    A, p, m, n, seed, L = _problem()
    st = oracle.Setup(A, p, m, n, seed)
    st.Y = np.ascontiguousarray(st.Y[:, c0: c0 + w])
    st.n = w
    return torch.from_numpy(oracle.sequence(A, st, L).astype(np.int64))


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, p, m, n, seed, L = _problem()
        S = shard.sharded_sequence(_oracle_slab, n, rank, world)
        np.save(out_path + ".%d.npy" % rank, S.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sequence_equals_whole_block(tmp_path, world):
    out = str(tmp_path / "S")
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    A, p, m, n, seed, L = _problem()
    ref = oracle.sequence(A, oracle.Setup(A, p, m, n, seed), L)
    for r in range(world):
        got = np.load(out + ".%d.npy" % r)
        assert got.shape == (L, m, n)
        assert np.array_equal(got.astype(np.uint32), ref), "rank %d" % r


def test_column_slab_partition():
    for n in range(1, 40):
        for world in range(1, n + 1):
            spans = [shard.column_slab(n, r, world) for r in range(world)]
            assert spans[0][0] == 0
            assert all(spans[r][0] + spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            assert spans[-1][0] + spans[-1][1] == n
            ws = [w for _, w in spans]
            assert max(ws) - min(ws) <= 1 and min(ws) >= 1
    with pytest.raises(ValueError):
        shard.column_slab(8, 8, 8)


# ---------------------------------------------------------------------------
# independent jobs (matrices x primes) dealt to ranks, ranks gathered
# ---------------------------------------------------------------------------

def _jobs():
    mats = [synth.planted_sparse(60 + 25 * i, 50 + 20 * i, 30 + 10 * i, row_len=4, seed=40 + i) for i in range(5)]
    primes = [65521, 1073741789, 2147483629]
    return mats, [(i, p) for i in range(len(mats)) for p in primes]


def _jobs_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mats, jobs = _jobs()
        share = shard.deal_jobs([mats[i].nnz for i, _ in jobs], world)[rank]
        ranks = [oracle.rank_sparse(mats[jobs[j][0]], jobs[j][1]) for j in share]
        allr = shard.gather_job_results(share, ranks, len(jobs), world)
        np.save(out_path + ".%d.npy" % rank, allr.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_jobs_dealt_and_gathered_in_job_order(tmp_path, world):
    out = str(tmp_path / "R")
    mp.start_processes(_jobs_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    mats, jobs = _jobs()
    for r in range(world):
        got = np.load(out + ".%d.npy" % r)
        assert got.tolist() == [mats[i].rank for i, _ in jobs], "rank %d" % r
        # rank over Q = the maximum over the primes
        for i, A in enumerate(mats):
            assert max(got[k] for k, (ii, _) in enumerate(jobs) if ii == i) == A.rank


def test_deal_jobs_balances_and_covers():
    costs = [5, 1, 1, 1, 1, 1, 3, 2, 8, 1]
    for world in [1, 2, 3, 4, 12]:
        share = shard.deal_jobs(costs, world)
        flat = sorted(j for s in share for j in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[j] for j in s) for s in share]
        if world <= len(costs):
            assert max(loads) - min(loads) <= max(costs)
    with pytest.raises(ValueError):
        shard.deal_jobs(costs, 0)
