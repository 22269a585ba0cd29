"""Batched jobs (wr_rank_batch) and the continuous-batching server: every
result in the mix is bit-identical to the same job run alone, admission
overlaps requests and respects the device-memory budget, and errors reach the
caller.  The exact-equality tolerance is the one that continuous batching
states for this method (results are exact residues)."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_0704_2351_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRIMES = [1073741789, 1073741783, 1073741741, 1073741723]


@pytest.fixture(scope="module")
def wr():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0704_2351_gb300 import _build
    _build.build()
    from paper_0704_2351_gb300 import wr as w
    return w


@pytest.fixture(scope="module")
def ctx(wr):
    c = wr.wr_create(0)
    yield c
    wr.wr_destroy(c)


def _load(wr, ctx, A):
    return wr.wr_matrix_load_csr(ctx, A.rows, A.cols, A.rowptr, A.colidx, A.vals)


def _result(wr, res, m, n):
    out = dict(rank=wr.wr_result_rank(res), **wr.wr_result_info(res))
    out["S"] = wr.wr_result_sequence(res, m, n)
    out["F"], out["delta"] = wr.wr_result_generator(res, n)
    wr.wr_result_free(res)
    return out


def _same(a, b):
    return (a["rank"] == b["rank"] and a["deg_det"] == b["deg_det"] and a["codeg"] == b["codeg"]
            and np.array_equal(a["S"], b["S"]) and np.array_equal(a["F"], b["F"])
            and np.array_equal(a["delta"], b["delta"]))


def _mix():
    """Matrices of uneven sizes (a chain-complex pair, planted matrices, a
    power-law one) with several primes, block widths and both projections."""
    d_n, d_n1 = synth.chain_pair(3000, seed=11, homology=2)
    mats = [d_n, d_n1,
            synth.planted_sparse(900, 700, 610, row_len=6, seed=5),
            synth.planted_sparse(4000, 4200, 3900, row_len=9, seed=6),
            synth.config1(scale=0.04)]
    jobs = []
    for i, A in enumerate(mats):
        for k, p in enumerate(PRIMES[: 2 + (i % 3)]):
            b = [4, 8, 16][(i + k) % 3]
            sym = (i + k) % 2 == 1
            jobs.append((i, p, b, 1000 + 10 * i + k, sym))
    return mats, jobs


def _params(wr, p, b, seed, sym):
    return wr.make_params(p, b, b, seed, want=3,
                          projection=wr.WR_PROJ_SYMMETRIC if sym else wr.WR_PROJ_GENERIC)


def test_rank_batch_matches_alone(wr, ctx):
    mats, jobs = _mix()
    handles = [_load(wr, ctx, A) for A in mats]
    alone = []
    t0 = time.perf_counter()
    for (i, p, b, seed, sym) in jobs:
        alone.append(_result(wr, wr.wr_rank(ctx, handles[i], _params(wr, p, b, seed, sym)), b, b))
    t_alone = time.perf_counter() - t0
    wr.wr_set_batch_slots(ctx, 6)
    t0 = time.perf_counter()
    outs = wr.wr_rank_batch(ctx, [handles[i] for (i, *_r) in jobs],
                            [_params(wr, p, b, seed, sym) for (i, p, b, seed, sym) in jobs])
    t_batch = time.perf_counter() - t0
    for j, (i, p, b, seed, sym) in enumerate(jobs):
        got = _result(wr, outs[j], b, b)
        assert _same(got, alone[j]), "job %d differs from the same job alone" % j
        assert got["rank"] == mats[i].rank
    print("alone %.3f s, batched %.3f s, %d jobs" % (t_alone, t_batch, len(jobs)))
    for h in handles:
        wr.wr_matrix_free(h)


def _heavy(R, C, seed):
    """A planted matrix plus a row and a column longer than one SELL segment
    (the split-row path of both passes)."""
    A = synth.planted_sparse(R, C, min(R, C) - 40, row_len=7, seed=seed)
    rng = np.random.default_rng(seed)
    r = [np.repeat(np.arange(R), np.diff(A.rowptr)), np.full(600, int(rng.integers(0, R))), rng.choice(R, 600, False)]
    c = [A.colidx.astype(np.int64), rng.choice(C, 600, False), np.full(600, int(rng.integers(0, C)))]
    v = [A.vals.astype(np.int64), np.ones(600, dtype=np.int64), -np.ones(600, dtype=np.int64)]
    return synth.csr_from_coo(R, C, np.concatenate(r), np.concatenate(c), np.concatenate(v))


@pytest.mark.parametrize("b,nprimes", [(8, 4), (8, 3), (4, 4), (3, 2), (16, 2), (16, 3), (2, 4)])
def test_rank_batch_fused_primes_match_alone(wr, ctx, b, nprimes):
    """Jobs on one matrix modulo several primes (the rank over Q) share one
    sequence loop in the batch: slices of one block of up to 64 columns, each
    reduced modulo its own prime.  Every result equals the same job alone and
    the batch with the fusion off, bit for bit; the chain pair's ranks are
    the planted ones for every prime."""
    d_n, _ = synth.chain_pair(2500, seed=b * 7 + nprimes, homology=1)
    mats = [d_n, _heavy(1500, 1400, b + nprimes)]
    handles = [_load(wr, ctx, A) for A in mats]
    jobs = [(i, p, 500 + 17 * i + k) for i in range(len(mats)) for k, p in enumerate(PRIMES[:nprimes])]
    params = [wr.make_params(p, b, b, seed, want=3) for (i, p, seed) in jobs]
    alone = [_result(wr, wr.wr_rank(ctx, handles[i], prm), b, b) for (i, _, _), prm in zip(jobs, params)]
    wr.wr_set_batch_slots(ctx, 3)
    try:
        for fuse in [True, False]:
            wr.wr_set_batch_fusion(ctx, fuse)
            outs = wr.wr_rank_batch(ctx, [handles[i] for (i, _, _) in jobs], params)
            for j, (i, p, seed) in enumerate(jobs):
                got = _result(wr, outs[j], b, b)
                assert _same(got, alone[j]), "job %d (fusion %s) differs from the same job alone" % (j, fuse)
            assert all(alone[j]["rank"] == mats[0].rank for j in range(nprimes))
    finally:
        wr.wr_set_batch_fusion(ctx, True)
        for h in handles:
            wr.wr_matrix_free(h)


def test_rank_batch_reports_a_failing_job(wr, ctx):
    A = synth.planted_sparse(300, 260, 200, row_len=5, seed=2)
    h = _load(wr, ctx, A)
    good = wr.make_params(PRIMES[0], 4, 4, 1)
    bad = wr.make_params(1073741790, 4, 4, 1)  # not prime
    with pytest.raises(wr.WrError) as ei:
        wr.wr_rank_batch(ctx, [h, h, h], [good, bad, good])
    assert ei.value.status == wr.WR_ENOTPRIME
    assert "batch job 1" in ei.value.message
    wr.wr_matrix_free(h)


def test_rank_batch_edge_cases(wr, ctx):
    assert wr.wr_rank_batch(ctx, [], []) == []
    Z = synth.csr_from_coo(6, 5, np.zeros(0), np.zeros(0), np.zeros(0))
    h = _load(wr, ctx, Z)
    outs = wr.wr_rank_batch(ctx, [h], [wr.make_params(PRIMES[1], 2, 2, 3)])
    assert wr.wr_result_rank(outs[0]) == 0
    wr.wr_result_free(outs[0])
    wr.wr_matrix_free(h)
    with pytest.raises(wr.WrError):
        wr.wr_set_batch_slots(ctx, 0)


def test_server_results_match_alone_with_overlap(wr, ctx):
    mats, jobs = _mix()
    handles = [_load(wr, ctx, A) for A in mats]
    alone = [_result(wr, wr.wr_rank(ctx, handles[i], _params(wr, p, b, seed, sym)), b, b)
             for (i, p, b, seed, sym) in jobs]
    srv = wr.wr_server_start(ctx, max_slots=4, hbm_budget=0, queue_cap=64)
    tickets = []

    def submit_all():
        # staggered arrivals: later requests arrive while earlier ones run
        for (i, p, b, seed, sym) in jobs:
            tickets.append(wr.wr_submit(srv, handles[i], _params(wr, p, b, seed, sym)))
            time.sleep(0.01)

    th = threading.Thread(target=submit_all)
    th.start()
    th.join()
    for j, t in enumerate(tickets):
        i, p, b, seed, sym = jobs[j]
        got = _result(wr, wr.wr_wait(srv, t, 600000), b, b)
        assert _same(got, alone[j]), "request %d differs from the same request alone" % j
    st = wr.wr_server_stats(srv)
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["max_resident"] >= 2, "no request was admitted while another one was resident"
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert st["kernel_launches"] > 0
    wr.wr_server_stop(srv)
    for h in handles:
        wr.wr_matrix_free(h)


def test_server_memory_admission(wr, ctx):
    A = synth.planted_sparse(2000, 1800, 1500, row_len=8, seed=9)
    h = _load(wr, ctx, A)
    prm = wr.make_params(PRIMES[2], 8, 8, 4)
    need = wr.wr_rank_device_bytes(ctx, h, prm)
    assert need > 4 * 2000 * 8
    # a budget that holds one request but not two: never two resident
    srv = wr.wr_server_start(ctx, max_slots=4, hbm_budget=int(need * 1.5), queue_cap=16)
    ts = [wr.wr_submit(srv, h, prm) for _ in range(4)]
    ranks = [wr.wr_result_rank(wr.wr_wait(srv, t, 600000)) for t in ts]
    assert ranks == [1500] * 4
    assert wr.wr_server_stats(srv)["max_resident"] == 1
    # a request above the budget is refused at submission
    big = wr.make_params(PRIMES[2], 32, 32, 4)
    assert wr.wr_rank_device_bytes(ctx, h, big) > int(need * 1.5)
    with pytest.raises(wr.WrError) as ei:
        wr.wr_submit(srv, h, big)
    assert ei.value.status == wr.WR_EINVAL
    with pytest.raises(wr.WrError) as ei:
        wr.wr_wait(srv, 10 ** 9, 10)
    assert ei.value.status == wr.WR_ETIMEDOUT
    wr.wr_server_stop(srv)
    wr.wr_matrix_free(h)


def test_memory_estimate_covers_pm_basis(wr, ctx):
    """The admission bound grows by the PM-Basis buffers (residual, bases,
    transform buffers) when the sigma-basis runs PM-Basis (q = 64, L > 2,048)
    and not when a leaf as long as the sequence keeps it on the M-Basis."""
    A = synth.planted_sparse(40000, 39000, 38000, row_len=4, seed=12)
    h = _load(wr, ctx, A)
    prm = wr.make_params(PRIMES[2], 32, 32, 4)
    L = 2 * -(-39000 // 32) + 2
    try:
        pm = wr.wr_rank_device_bytes(ctx, h, prm)
        wr.wr_set_sigma_leaf(ctx, L + 10)
        mb = wr.wr_rank_device_bytes(ctx, h, prm)
    finally:
        wr.wr_set_sigma_leaf(ctx, 0)
        wr.wr_matrix_free(h)
    q = 64
    Lz = 1 << (L - 1).bit_length()
    assert pm - mb >= 4 * L * 32 * q + 3 * 4 * (L // 2) * q * q + 4 * 5 * q * q * Lz


def test_server_refuses_invalid_requests_and_keeps_serving(wr, ctx):
    A = synth.planted_sparse(200, 180, 150, row_len=4, seed=3)
    h = _load(wr, ctx, A)
    srv = wr.wr_server_start(ctx, max_slots=2, hbm_budget=0, queue_cap=8)
    with pytest.raises(wr.WrError) as ei:
        wr.wr_submit(srv, h, wr.make_params(1073741790, 2, 2, 1))
    assert ei.value.status == wr.WR_ENOTPRIME
    ok = wr.wr_submit(srv, h, wr.make_params(PRIMES[3], 2, 2, 1))
    assert wr.wr_result_rank(wr.wr_wait(srv, ok, 600000)) == 150
    st = wr.wr_server_stats(srv)
    assert (st["submitted"], st["completed"], st["failed"]) == (1, 1, 0)
    wr.wr_server_stop(srv)
    wr.wr_matrix_free(h)
    assert oracle.rank_sparse(A, PRIMES[3]) == 150


def test_torch_caching_allocator_owns_the_device_memory(wr, ctx):
    """With wr_set_allocator every device buffer of the library (matrix
    layouts, sequence state, sigma-basis, batch slots) comes from PyTorch's
    caching allocator and goes back to it; the results do not change."""
    counts = {"alloc": 0, "free": 0}

    def alloc(nbytes, stream):
        counts["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(nbytes, device=0, stream=stream)

    def release(ptr, nbytes, stream):
        counts["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    A = synth.planted_sparse(1500, 1400, 1200, row_len=7, seed=21)
    c2 = wr.wr_create(0)
    try:
        wr.wr_set_allocator(c2, alloc, release)
        h = _load(wr, c2, A)
        prm = [_params(wr, PRIMES[k], 8, 50 + k, k == 1) for k in range(3)]
        got = [_result(wr, wr.wr_rank(c2, h, prm[0]), 8, 8)]
        got += [_result(wr, o, 8, 8) for o in wr.wr_rank_batch(c2, [h, h], prm[1:])]
        wr.wr_matrix_free(h)
        assert counts["alloc"] > 0 and counts["alloc"] == counts["free"]
    finally:
        wr.wr_destroy(c2)
    h0 = _load(wr, ctx, A)
    for g, p in zip(got, prm):
        assert _same(g, _result(wr, wr.wr_rank(ctx, h0, p), 8, 8))
        assert g["rank"] == 1200
    wr.wr_matrix_free(h0)
    with pytest.raises(wr.WrError):
        wr.wr_set_allocator(ctx, alloc, None)
