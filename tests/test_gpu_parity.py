"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work, so the bar is bit-exactness: sequences, sigma-bases, generator
degrees, valuations and ranks must equal the oracle's.  Sizes span several
SELL chunks, split (heavy) rows, ragged tails and padded block widths.
"""
import numpy as np
import pytest

import oracle
from paper_0704_2351_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRIMES = [65521, 1073741789, 2147483629]


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


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def from_dev(t):
    return t.cpu().numpy().view(np.uint32)


def heavy_matrix(R, C, seed, heavy=3, heavy_len=700, per_row=5):
    """Random sparse matrix plus a few rows and columns longer than one SELL
    segment (256 entries), to exercise the split-row path in both passes."""
    rng = np.random.default_rng(seed)
    base = synth.random_sparse(R, C, per_row, seed=seed)
    r = [np.repeat(np.arange(R), np.diff(base.rowptr))]
    c = [base.colidx.astype(np.int64)]
    v = [base.vals.astype(np.int64)]
    for _ in range(heavy):
        row = int(rng.integers(0, R))
        cols = rng.choice(C, size=min(heavy_len, C), replace=False)
        r.append(np.full(len(cols), row)); c.append(cols); v.append(rng.choice([-1, 1, 2, -3], size=len(cols)))
        col = int(rng.integers(0, C))
        rows = rng.choice(R, size=min(heavy_len, R), replace=False)
        r.append(rows); c.append(np.full(len(rows), col)); v.append(rng.choice([-1, 1, 3], size=len(rows)))
    return synth.csr_from_coo(R, C, np.concatenate(r), np.concatenate(c), np.concatenate(v))


def load(wr, ctx, A):
    return wr.wr_matrix_load_csr(ctx, A.rows, A.cols, A.rowptr, A.colidx, A.vals)


# ------------------------------------------------------------------ black box (A4, A5)

@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("width", [1, 3, 8, 16, 32])
def test_blackbox_parity(wr, ctx, p, side, width):
    A = heavy_matrix(1100, 900, seed=width * 7 + side)
    mat = load(wr, ctx, A)
    seed = 99 + width
    N = A.cols if side == 0 else A.rows
    Mo = A.rows if side == 0 else A.cols
    rng = np.random.default_rng(width)
    v = rng.integers(0, p, size=(N, width)).astype(np.uint32)
    prm = wr.make_params(p, 1, width, seed, side=side)
    dout = torch.empty((N, width), dtype=torch.int32, device="cuda")
    wr.wr_blackbox_apply_device(ctx, mat, prm, to_dev(v), dout, width)
    d1 = oracle.derive_diag(seed, oracle.TAG_D1, N, p)
    d2 = oracle.derive_diag(seed, oracle.TAG_D2, Mo, p)
    ref = oracle.blackbox_apply(A, p, side, d1, d2, v)
    assert np.array_equal(from_dev(dout), ref)
    wr.wr_matrix_free(mat)


def test_blackbox_tiny_and_ragged(wr, ctx):
    p = 65521
    for (R, C, k) in [(1, 1, 1), (3, 70, 2), (33, 31, 4), (65, 2, 1)]:
        A = synth.random_sparse(R, C, k, seed=R * C)
        mat = load(wr, ctx, A)
        for side in [0, 1]:
            N = A.cols if side == 0 else A.rows
            Mo = A.rows if side == 0 else A.cols
            v = np.random.default_rng(1).integers(0, p, size=(N, 2)).astype(np.uint32)
            prm = wr.make_params(p, 1, 2, 5, side=side)
            dout = torch.empty((N, 2), dtype=torch.int32, device="cuda")
            wr.wr_blackbox_apply_device(ctx, mat, prm, to_dev(v), dout, 2)
            ref = oracle.blackbox_apply(A, p, side, oracle.derive_diag(5, 3, N, p),
                                        oracle.derive_diag(5, 4, Mo, p), v)
            assert np.array_equal(from_dev(dout), ref)
        wr.wr_matrix_free(mat)


def _wide_matrix(seed, R=700, C=640):
    """heavy_matrix with most values multiplied up to the int16 range."""
    A = heavy_matrix(R, C, seed=seed, heavy=2, heavy_len=400)
    rng = np.random.default_rng(seed)
    v = A.vals.astype(np.int64) * rng.choice([1, 97, 1021, 10007], size=A.nnz)
    v = np.clip(v, -32767, 32767).astype(np.int32)
    return synth.CSR(A.rows, A.cols, A.rowptr, A.colidx, v)


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("p", [65521, 2147483629])
def test_wide_values_blackbox_and_sequence(wr, ctx, side, p):
    """Entries up to +-32767 (the int16 layout): one application on both
    sides against the oracle, and the sequence."""
    A = _wide_matrix(60 + side)
    assert np.abs(A.vals).max() > 127
    mat = load(wr, ctx, A)
    N = A.cols if side == 0 else A.rows
    M = A.rows if side == 0 else A.cols
    rng = np.random.default_rng(side)
    v = rng.integers(0, p, size=(N, 4)).astype(np.uint32)
    dout = torch.empty((N, 4), dtype=torch.int32, device="cuda")
    wr.wr_blackbox_apply_device(ctx, mat, wr.make_params(p, 1, 4, 9, side=side), to_dev(v), dout, 4)
    ref = oracle.blackbox_apply(A, p, side, oracle.derive_diag(9, 3, N, p), oracle.derive_diag(9, 4, M, p), v)
    assert np.array_equal(from_dev(dout), ref)
    wr.wr_matrix_free(mat)
    st = oracle.Setup(A, p, 4, 4, seed=3, side=side)
    assert np.array_equal(gpu_sequence(wr, ctx, A, p, 4, 4, 3, 120, side=side), oracle.sequence(A, st, 120))


def test_wide_values_rank_and_limits(wr, ctx):
    p = 1073741789
    A = synth.planted_sparse(800, 700, 560, row_len=6, seed=19)
    B = synth.CSR(A.rows, A.cols, A.rowptr, A.colidx, (A.vals * 257).astype(np.int32))  # rank kept for p != 257
    assert np.abs(B.vals).max() > 127
    assert gpu_rank(wr, ctx, B, p, 4, 4, 2)["rank"] == 560
    # a wide matrix with a column of 65,536 entries is refused
    R = 65536
    rows = np.arange(R)
    cols = np.zeros(R, dtype=np.int64)
    vals = np.ones(R, dtype=np.int64)
    vals[0] = 200
    L = synth.csr_from_coo(R, 2, rows, cols, vals)
    with pytest.raises(wr.WrError) as ei:
        load(wr, ctx, L)
    assert ei.value.status == wr.WR_EOVERFLOW
    # the same column with small values is fine
    vals[0] = 1
    mat = load(wr, ctx, synth.csr_from_coo(R, 2, rows, cols, vals))
    wr.wr_matrix_free(mat)


# ------------------------------------------------------------------ sequence (A2, A3, A6, A7)

def gpu_sequence(wr, ctx, A, p, m, n, seed, L, side=-1, symmetric=False):
    mat = load(wr, ctx, A)
    prm = wr.make_params(p, m, n, seed, side=side,
                         projection=wr.WR_PROJ_SYMMETRIC if symmetric else wr.WR_PROJ_GENERIC)
    dS = torch.empty((L, m, n), dtype=torch.int32, device="cuda")
    wr.wr_sequence_device(ctx, mat, prm, dS, L)
    S = from_dev(dS)
    wr.wr_matrix_free(mat)
    return S


def test_sequence_config0_scalar_full(wr, ctx):
    A = synth.config0()
    p = synth.PRIME_C0
    st = oracle.Setup(A, p, 1, 1, seed=synth.SEED_BASE)
    L = oracle.seq_length(st.N, 1, 1)
    S_ref = oracle.sequence(A, st, L)
    S = gpu_sequence(wr, ctx, A, p, 1, 1, synth.SEED_BASE, L)
    assert np.array_equal(S, S_ref)


@pytest.mark.parametrize("m,n", [(2, 2), (3, 5), (8, 8), (4, 16), (32, 32), (1, 7)])
@pytest.mark.parametrize("p", [65521, 2147483629])
def test_sequence_block_parity(wr, ctx, m, n, p):
    A = heavy_matrix(700, 620, seed=m * 100 + n, heavy=2, heavy_len=400)
    st = oracle.Setup(A, p, m, n, seed=3)
    L = min(oracle.seq_length(st.N, m, n), 300)
    S_ref = oracle.sequence(A, st, L)
    S = gpu_sequence(wr, ctx, A, p, m, n, 3, L)
    assert np.array_equal(S, S_ref)


@pytest.mark.parametrize("side", [0, 1])
def test_sequence_sides_and_symmetric(wr, ctx, side):
    p = 1073741789
    A = heavy_matrix(500, 560, seed=17 + side, heavy=2, heavy_len=300)
    for sym in [False, True]:
        st = oracle.Setup(A, p, 4, 4, seed=21, side=side, symmetric=sym)
        S_ref = oracle.sequence(A, st, 150)
        S = gpu_sequence(wr, ctx, A, p, 4, 4, 21, 150, side=side, symmetric=sym)
        assert np.array_equal(S, S_ref)
        if sym:
            assert all(np.array_equal(S[i], S[i].T) for i in range(len(S)))


@pytest.mark.parametrize("n,L,side", [(1, 41, 0), (1, 40, 1), (8, 97, 0), (8, 96, 1), (32, 33, 0), (4, 1, 0),
                                      (4, 2, 1), (4, 3, 0)])
@pytest.mark.parametrize("p", [65521, 2147483629])
def test_sequence_symmetric_two_terms_per_application(wr, ctx, n, L, side, p):
    """X = Y: the GPU takes S_2k = V_k^T V_k and S_2k+1 = (A D1 V_k)^T D2 (A D1 V_k)
    from one application of A~ per two terms; the oracle applies A~ once per
    term.  Odd and even L (the last application's second term is dropped when
    it would be S_L), L = 1 and 2, and both sides."""
    A = heavy_matrix(640, 590, seed=n * 7 + L, heavy=2, heavy_len=350)
    st = oracle.Setup(A, p, n, n, seed=40 + n, side=side, symmetric=True)
    S_ref = oracle.sequence(A, st, L)
    S = gpu_sequence(wr, ctx, A, p, n, n, 40 + n, L, side=side, symmetric=True)
    assert np.array_equal(S, S_ref)


@pytest.mark.parametrize("n,L,side", [(1, 41, 0), (1, 40, 1), (3, 57, 0), (8, 97, 0), (8, 96, 1), (16, 33, 1),
                                      (4, 1, 0), (4, 2, 1), (4, 3, 0), (32, 65, 0), (32, 64, 1), (24, 29, 1)])
@pytest.mark.parametrize("p", [65521, 2147483629])
def test_sequence_generic_paired_two_terms_per_application(wr, ctx, n, L, side, p):
    """Generic projection with m = n: the GPU carries [D1 X | D1 Y] as one
    block and takes S_2k = U_k^T V_k and S_2k+1 = (A D1 U_k)^T D2 (A D1 V_k)
    from one application per two terms; the oracle applies A~ to Y once per
    term.  The sequence is the same with the pairing switched off.  Odd and
    even L, L = 1, 2, 3, a padded block width (n = 3) and both sides."""
    A = heavy_matrix(610, 575, seed=n * 11 + L, heavy=2, heavy_len=330)
    st = oracle.Setup(A, p, n, n, seed=60 + n, side=side)
    S_ref = oracle.sequence(A, st, L)
    S = gpu_sequence(wr, ctx, A, p, n, n, 60 + n, L, side=side)
    assert np.array_equal(S, S_ref)
    try:
        wr.wr_set_paired_projection(ctx, False)
        assert np.array_equal(gpu_sequence(wr, ctx, A, p, n, n, 60 + n, L, side=side), S_ref)
    finally:
        wr.wr_set_paired_projection(ctx, True)


@pytest.mark.parametrize("m,n,sym,chunk", [(8, 8, False, 0), (8, 8, True, 5), (3, 3, False, 64), (4, 7, False, 13),
                                            (1, 1, False, 0), (16, 16, True, 0)])
def test_rank_pipeline_matches_sequential(wr, ctx, m, n, sym, chunk):
    """wr_rank with the sigma-basis trailing the sequence on a second stream
    (the default) gives the same sequence, generator and rank as the phases
    run one after the other, and both equal the oracle's; chunk sizes that are
    not a multiple of the window's order tile make the trailing windows wait
    for rounded-up term counts."""
    p = 1073741789
    A = synth.planted_sparse(1300, 1150, 1020, row_len=7, seed=m * 31 + n + chunk)
    try:
        wr.wr_set_sigma_chunk(ctx, chunk)
        got = gpu_rank(wr, ctx, A, p, m, n, 77, want=3, symmetric=sym)
        wr.wr_set_pipeline(ctx, False)
        seq = gpu_rank(wr, ctx, A, p, m, n, 77, want=3, symmetric=sym)
    finally:
        wr.wr_set_pipeline(ctx, True)
        wr.wr_set_sigma_chunk(ctx, 0)
    assert got["rank"] == seq["rank"] == 1020
    assert np.array_equal(got["S"], seq["S"]) and np.array_equal(got["F"], seq["F"])
    ref = oracle.rank_wiedemann(A, p, m, n, seed=77, symmetric=sym)
    assert np.array_equal(got["S"], ref["S"]) and np.array_equal(got["F"], ref["F"])


@pytest.mark.parametrize("m,leaf,R,C,r", [(4, 64, 1300, 1150, 1020), (8, 64, 1300, 1150, 900),
                                          (32, 64, 4400, 4200, 4000), (20, 64, 3000, 2900, 2700)])
def test_rank_pipeline_pm_segments(wr, ctx, m, leaf, R, C, r):
    """PM-Basis trailing the sequence in segments (each about half of the
    orders still to come, down to two leaves; leaves forced short so that a
    small case has several segments, wide blocks included): the same
    generator and rank as PM-Basis on the whole sequence, and both equal the
    oracle's."""
    p = 2147483629
    A = synth.planted_sparse(R, C, r, row_len=6, seed=m * 7 + leaf)
    try:
        wr.wr_set_sigma_leaf(ctx, leaf)
        got = gpu_rank(wr, ctx, A, p, m, m, 5, want=3)
        wr.wr_set_pipeline(ctx, 2)  # the sigma-basis's stream first
        got2 = gpu_rank(wr, ctx, A, p, m, m, 5, want=3)
        wr.wr_set_pipeline(ctx, 3)  # the sequence's stream first
        got3 = gpu_rank(wr, ctx, A, p, m, m, 5, want=3)
        wr.wr_set_pipeline(ctx, False)
        seq = gpu_rank(wr, ctx, A, p, m, m, 5, want=3)
        for bad in [4, -1]:
            with pytest.raises(wr.WrError):
                wr.wr_set_pipeline(ctx, bad)
    finally:
        wr.wr_set_pipeline(ctx, True)
        wr.wr_set_sigma_leaf(ctx, 0)
    assert got["rank"] == seq["rank"] == got2["rank"] == got3["rank"] == r
    for g in [got, got2, got3]:
        assert np.array_equal(g["S"], seq["S"]) and np.array_equal(g["F"], seq["F"])
    ref = oracle.rank_wiedemann(A, p, m, m, seed=5)
    assert np.array_equal(got["F"], ref["F"]) and got["rank"] == ref["rank"]


@pytest.mark.parametrize("m,sym,chunk,quiet,R,C,r", [(4, False, 0, 64, 2100, 2000, 600),
                                                       (8, True, 0, 64, 3000, 2600, 1200),
                                                       (4, False, 16, 48, 1800, 1700, 400),
                                                       (1, False, 0, 64, 900, 800, 300),
                                                       (2, False, 0, 128, 1500, 1400, 1400)])
def test_rank_early_termination(wr, ctx, m, sym, chunk, quiet, R, C, r):
    """Early termination: the trailing M-Basis stops the sequence once the
    generator candidates have been quiet for `quiet` orders.  The rank equals
    the planted one, the generator equals the oracle's from all L terms (and
    from the terms actually used), the terms used match the oracle's, and a
    rank-deficient matrix needs far fewer than L terms (about 2r/n + O(1));
    a full-rank one (last case) runs to the end or close to it."""
    p = 1073741789
    A = synth.planted_sparse(R, C, r, row_len=6, seed=r + m)
    L = oracle.seq_length(min(R, C), m, m)
    try:
        wr.wr_set_sigma_chunk(ctx, chunk)
        wr.wr_set_early_termination(ctx, quiet)
        got = gpu_rank(wr, ctx, A, p, m, m, 91, want=3, symmetric=sym)
    finally:
        wr.wr_set_early_termination(ctx, 0)
        wr.wr_set_sigma_chunk(ctx, 0)
    used = got["seq_len"]
    assert got["rank"] == r
    assert 0 < used <= L and got["S"].shape[0] == used
    ref = oracle.rank_wiedemann(A, p, m, m, seed=91, symmetric=sym)
    assert np.array_equal(got["S"], ref["S"][:used])
    assert np.array_equal(got["F"], ref["F"]) and np.array_equal(got["delta"], ref["delta"])
    short = oracle.rank_wiedemann(A, p, m, m, seed=91, symmetric=sym, L=used)
    assert short["rank"] == r and np.array_equal(short["F"], got["F"])
    if r < min(R, C) // 2:
        assert used < L - (min(R, C) - r) // (2 * m), "early termination saved too little (%d of %d)" % (used, L)
    with pytest.raises(wr.WrError):
        wr.wr_set_early_termination(ctx, -1)


def test_rank_with_chain_reduction(wr, ctx):
    """Loads with the chain reduction: wr_rank = pivots taken + rank of the
    reduced matrix = the planted rank (and the oracle's elimination rank);
    the reduction agrees with the host entry point; device-side loads reduce
    the same way; a matrix that reduces to nothing has rank = its pivots."""
    p = 1073741789
    d_n, d_n1 = synth.chain_pair(2500, seed=5, homology=2)
    mats = [synth.planted_sparse(1500, 1300, 1111, row_len=6, seed=12), d_n, d_n1,
            synth.config1(scale=0.03)]
    n = 40
    bid = synth.dense_to_csr(np.eye(n, dtype=np.int64) + np.diag(-np.ones(n - 1, dtype=np.int64), 1))
    bid.rank = n
    mats.append(bid)
    try:
        wr.wr_set_chain_reduction(ctx, True)
        for A in mats:
            h = load(wr, ctx, A)
            red = wr.wr_matrix_reduction(h)
            r, c, *_rest, off = wr.wr_chain_reduce_csr(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
            assert (red["rows_in"], red["cols_in"], red["rank_offset"]) == (A.rows, A.cols, off)
            info = wr.wr_matrix_info(h)
            assert (info["rows"], info["cols"]) == (r, c)
            for b, sym in [(8, False), (4, True)]:
                res = wr.wr_rank(ctx, h, wr.make_params(p, b, b, 3, projection=wr.WR_PROJ_SYMMETRIC if sym
                                                      else wr.WR_PROJ_GENERIC))
                assert wr.wr_result_rank(res) == A.rank
                wr.wr_result_free(res)
            wr.wr_matrix_free(h)
            # the same from device arrays
            d_rp = torch.from_numpy(A.rowptr.astype(np.int64)).cuda()
            d_ci = torch.from_numpy(A.colidx.astype(np.int32)).cuda()
            d_va = torch.from_numpy(A.vals.astype(np.int32)).cuda()
            h = wr.wr_matrix_load_csr_device(ctx, A.rows, A.cols, A.nnz, d_rp, d_ci, d_va)
            assert wr.wr_matrix_reduction(h)["rank_offset"] == off
            res = wr.wr_rank(ctx, h, wr.make_params(p, 8, 8, 4))
            assert wr.wr_result_rank(res) == A.rank
            wr.wr_result_free(res)
            wr.wr_matrix_free(h)
    finally:
        wr.wr_set_chain_reduction(ctx, False)
    assert oracle.rank_sparse(mats[0], p) == mats[0].rank


def test_locality_order_changes_nothing_at_the_boundary(wr, ctx):
    """Loads with the locality order renumber rows and columns by decreasing
    entry count; X, Y, D1, D2 are drawn at the loaded indices, so sequences
    (generic, paired, symmetric, both sides, column slabs), black-box
    applications (allocating and allocation-free) and ranks equal the
    oracle's and those of the unordered load."""
    p = 1073741789
    A = heavy_matrix(1200, 1000, seed=71, heavy=3, heavy_len=600)
    P = synth.config1(scale=0.02)
    try:
        wr.wr_set_locality_order(ctx, True)
        for side in [0, 1]:
            for (m, n, sym) in [(4, 4, False), (3, 5, False), (8, 8, True), (1, 1, False)]:
                st = oracle.Setup(A, p, m, n, seed=13, side=side, symmetric=sym)
                S_ref = oracle.sequence(A, st, 90)
                assert np.array_equal(gpu_sequence(wr, ctx, A, p, m, n, 13, 90, side=side, symmetric=sym), S_ref)
            N = A.cols if side == 0 else A.rows
            Mo = A.rows if side == 0 else A.cols
            v = np.random.default_rng(side).integers(0, p, size=(N, 8)).astype(np.uint32)
            d1 = oracle.derive_diag(21, oracle.TAG_D1, N, p)
            d2 = oracle.derive_diag(21, oracle.TAG_D2, Mo, p)
            ref = oracle.blackbox_apply(A, p, side, d1, d2, v)
            mat = load(wr, ctx, A)
            prm = wr.make_params(p, 1, 8, 21, side=side)
            dout = torch.empty((N, 8), dtype=torch.int32, device="cuda")
            wr.wr_blackbox_apply_device(ctx, mat, prm, to_dev(v), dout, 8)
            assert np.array_equal(from_dev(dout), ref)
            dout2 = torch.empty((N, 8), dtype=torch.int32, device="cuda")
            wr.wr_blackbox_apply_device_noalloc(ctx, mat, prm, to_dev(v), dout2, 8)
            assert np.array_equal(from_dev(dout2), ref)
            wr.wr_matrix_free(mat)
        g = gpu_rank(wr, ctx, P, p, 8, 8, 5, want=3)
        wr.wr_set_chain_reduction(ctx, True)
        g2 = gpu_rank(wr, ctx, P, p, 8, 8, 5)
    finally:
        wr.wr_set_locality_order(ctx, False)
        wr.wr_set_chain_reduction(ctx, False)
    ref = oracle.rank_wiedemann(P, p, 8, 8, seed=5)
    assert g["rank"] == ref["rank"] == P.rank == g2["rank"]
    assert np.array_equal(g["S"], ref["S"]) and np.array_equal(g["F"], ref["F"])


@pytest.mark.parametrize("m", [1, 4, 8])
def test_rank_planted_symmetric(wr, ctx, m):
    p = 1073741789
    for t in range(3):
        rng = np.random.default_rng(t * 17 + m)
        R, C = int(rng.integers(60, 500)), int(rng.integers(60, 500))
        r = int(rng.integers(1, min(R, C)))
        A = synth.planted_sparse(R, C, r, row_len=int(rng.integers(3, 9)), seed=t + 300 * m)
        ref = oracle.rank_wiedemann(A, p, m, m, seed=t, symmetric=True)
        g = gpu_rank(wr, ctx, A, p, m, m, t, want=3, symmetric=True)
        assert g["rank"] == ref["rank"] == r
        assert np.array_equal(g["S"], ref["S"])
        assert np.array_equal(g["F"], ref["F"])


@pytest.mark.parametrize("sym", [False, True])
def test_sequence_column_slabs_concatenate_to_the_whole(wr, ctx, sym):
    """Column slabs of Y (the multi-GPU split, computed here one after the
    other on one GPU): uneven widths, concatenated in column order, equal the
    whole sequence; each slab equals the oracle on its slab of Y."""
    p, m, n, seed, L = 1073741789, 8, 8, 12, 90
    A = heavy_matrix(520, 480, seed=23, heavy=2, heavy_len=260)
    mat = load(wr, ctx, A)
    prm = wr.make_params(p, m, n, seed,
                         projection=wr.WR_PROJ_SYMMETRIC if sym else wr.WR_PROJ_GENERIC)
    st = oracle.Setup(A, p, m, n, seed, symmetric=sym)
    S_ref = oracle.sequence(A, st, L)
    parts = []
    for c0, w in [(0, 3), (3, 1), (4, 4)]:
        d = torch.empty((L, m, w), dtype=torch.int32, device="cuda")
        wr.wr_sequence_slab_device(ctx, mat, prm, c0, w, d, L)
        parts.append(from_dev(d).reshape(L, m, w))
    assert np.array_equal(np.concatenate(parts, axis=2), S_ref)
    with pytest.raises(wr.WrError):
        wr.wr_sequence_slab_device(ctx, mat, prm, 6, 3, torch.empty((L, m, 3), dtype=torch.int32,
                                                                   device="cuda"), L)
    wr.wr_matrix_free(mat)


def test_sharded_sequence_single_rank_gpu(wr, ctx):
    """The shard module's GPU slab function with a one-rank gloo group."""
    import torch.distributed as dist
    from paper_0704_2351_gb300 import shard
    import socket
    s = socket.socket(); s.bind(("127.0.0.1", 0)); port = s.getsockname()[1]; s.close()
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    try:
        p, m, n, seed, L = 65521, 4, 6, 3, 40
        A = heavy_matrix(300, 280, seed=5, heavy=1, heavy_len=120)
        mat = load(wr, ctx, A)
        prm = wr.make_params(p, m, n, seed)
        f = shard.gpu_slab(ctx, mat, prm, L)
        S = shard.sharded_sequence(lambda c0, w: f(c0, w).cpu(), n, 0, 1)
        ref = oracle.sequence(A, oracle.Setup(A, p, m, n, seed), L)
        assert np.array_equal(S.numpy().view(np.uint32), ref)
        wr.wr_matrix_free(mat)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("m,n,sym,side", [(8, 8, False, 0), (8, 8, False, 1), (4, 4, True, 0), (3, 5, False, 1),
                                          (32, 32, False, 0), (1, 1, False, 1)])
@pytest.mark.parametrize("slab_bytes,wide", [(4096, False), (20000, False), (12000, True)])
def test_sequence_with_column_slabs(wr, ctx, m, n, sym, side, slab_bytes, wide):
    """Passes split into column slabs (several launches, each adding its exact
    row sums mod p to the output rows, the last applying the diagonal): the
    sequence and one black-box application equal the oracle's, with rows
    longer than a segment (split rows) cut across slabs, both sides, the
    paired, symmetric and unpaired projections."""
    p = 2147483629
    A = heavy_matrix(900, 820, seed=m * 31 + n + side, heavy=3, heavy_len=600)
    if wide:  # entries beyond int8: the layout with int16 values beside the columns
        A = synth.CSR(A.rows, A.cols, A.rowptr, A.colidx, (A.vals * 257).astype(np.int32))
    st = oracle.Setup(A, p, m, n, seed=13, side=side, symmetric=sym)
    L = 41
    S_ref = oracle.sequence(A, st, L)
    wr.wr_set_column_slabs(ctx, slab_bytes)  # before the loads: the matrices keep their CSR for the slabs
    try:
        assert np.array_equal(gpu_sequence(wr, ctx, A, p, m, n, 13, L, side=side, symmetric=sym), S_ref)
        mat = load(wr, ctx, A)
        v = np.random.default_rng(3).integers(0, p, size=(st.N, n)).astype(np.uint32)
        dout = torch.empty((st.N, n), dtype=torch.int32, device="cuda")
        wr.wr_blackbox_apply_device(ctx, mat, wr.make_params(p, 1, n, 13, side=side), to_dev(v), dout, n)
        assert np.array_equal(from_dev(dout), oracle.blackbox_apply(A, p, st.side, st.D1, st.D2, v))
        wr.wr_matrix_free(mat)
    finally:
        wr.wr_set_column_slabs(ctx, 0)


@pytest.mark.parametrize("m,n,sym,side,L", [(8, 8, False, 0, 331), (8, 8, True, 1, 300), (32, 32, True, 0, 261),
                                            (32, 32, False, 1, 140), (16, 16, True, 0, 2), (4, 4, False, 0, 3)])
def test_projection_overlap_gives_the_same_sequence(wr, ctx, m, n, sym, side, L):
    """The Gram projections beside the passes (side stream, forked and joined
    around each pass, captured into the 64-application graphs) give the
    oracle's sequence, as with the projections after the passes: lengths with
    several captured groups and an eager tail, odd and even L, L = 2 and 3."""
    p = 2147483629
    A = heavy_matrix(1200, 1100, seed=m + 3 * side + (7 if sym else 0), heavy=2, heavy_len=500)
    st = oracle.Setup(A, p, m, n, seed=21, side=side, symmetric=sym)
    S_ref = oracle.sequence(A, st, L)
    try:
        for on in [True, False]:
            wr.wr_set_projection_overlap(ctx, on)
            assert np.array_equal(gpu_sequence(wr, ctx, A, p, m, n, 21, L, side=side, symmetric=sym), S_ref), on
    finally:
        wr.wr_set_projection_overlap(ctx, False)


@pytest.mark.parametrize("m,n", [(1, 1), (2, 2), (4, 8), (4, 32), (32, 32)])
def test_lane_widths_give_identical_sequences(wr, ctx, m, n):
    """Every SpMM lane width (1, 2, 4, 8 residues per lane where it divides
    the block width, at most 32 lanes per row) gives the oracle's sequence;
    the autotuner only picks among them.  m = n = 32 runs the paired block of
    width 64."""
    p, seed, L = 2147483629, 5, 40
    A = heavy_matrix(900, 820, seed=41 + n, heavy=3, heavy_len=500)
    st = oracle.Setup(A, p, m, n, seed)
    S_ref = oracle.sequence(A, st, L)
    try:
        for wl in [1, 2, 4, 8]:
            if wl > n or n % wl:
                continue
            for hints in [0, 16]:  # plain and streaming cache hints
                wr.wr_set_lane_width(ctx, wl | hints)
                assert np.array_equal(gpu_sequence(wr, ctx, A, p, m, n, seed, L), S_ref), "lane width %d" % (wl | hints)
    finally:
        wr.wr_set_lane_width(ctx, 0)
    for bad in [3, 32, 19]:
        with pytest.raises(wr.WrError):
            wr.wr_set_lane_width(ctx, bad)


# ------------------------------------------------------------------ sigma-basis (A8)

def gpu_sigma(wr, ctx, S, p):
    L, m, n = S.shape
    q = m + n
    Dcap = L + 1
    dP = torch.empty(((Dcap + 1), n, q), dtype=torch.int32, device="cuda")
    ddeg = torch.empty(q, dtype=torch.int32, device="cuda")
    wr.wr_sigma_basis_device(ctx, to_dev(S), L, m, n, p, dP, ddeg, Dcap)
    return from_dev(dP), ddeg.cpu().numpy()


@pytest.mark.parametrize("m,n,L", [(1, 1, 50), (2, 3, 77), (3, 2, 130), (8, 8, 200), (5, 5, 65),
                                   (16, 16, 70), (32, 32, 40), (24, 20, 61), (32, 16, 50), (17, 32, 45),
                                   (32, 31, 39), (32, 1, 90)])
@pytest.mark.parametrize("p", [65521, 2147483629])
def test_sigma_basis_random_sequence(wr, ctx, m, n, L, p):
    rng = np.random.default_rng(m * 1000 + n * 10 + L)
    S = rng.integers(0, p, size=(L, m, n)).astype(np.uint32)
    M, deg = oracle.mbasis(S, p)
    P, dg = gpu_sigma(wr, ctx, S, p)
    assert np.array_equal(dg, deg)
    D = M.shape[0] - 1
    assert np.array_equal(P[: D + 1], M[:, :n, :])
    assert not P[D + 1:].any()


@pytest.mark.parametrize("m,n", [(1, 1), (4, 4), (2, 6), (20, 24), (32, 32)])
def test_sigma_basis_wiedemann_sequence(wr, ctx, m, n):
    """Structured (rank-deficient) sequences: degenerate discrepancies."""
    p = 65521
    A = synth.planted_sparse(300, 260, 170, row_len=5, seed=m + n)
    st = oracle.Setup(A, p, m, n, seed=4)
    S = oracle.sequence(A, st)
    M, deg = oracle.mbasis(S, p)
    P, dg = gpu_sigma(wr, ctx, S, p)
    assert np.array_equal(dg, deg)
    assert np.array_equal(P[: M.shape[0]], M[:, :n, :])


@pytest.mark.parametrize("chunk", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("p", [65521, 2147483629])
def test_sigma_basis_wide_chunks(wr, ctx, chunk, p):
    """Wide blocks (q = 64 and q = 45) with the chunk length forced: every
    chunk length up to the largest that fits, and ragged last chunks."""
    for m, n, L in [(32, 32, 37), (25, 20, 43)]:
        rng = np.random.default_rng(m * 100 + chunk)
        S = rng.integers(0, p, size=(L, m, n)).astype(np.uint32)
        M, deg = oracle.mbasis(S, p)
        wr.wr_set_sigma_chunk(ctx, chunk)
        try:
            P, dg = gpu_sigma(wr, ctx, S, p)
        finally:
            wr.wr_set_sigma_chunk(ctx, 0)
        assert np.array_equal(dg, deg)
        D = M.shape[0] - 1
        assert np.array_equal(P[: D + 1], M[:, :n, :])
        assert not P[D + 1:].any()


def test_sigma_basis_wide_rank_deficient_discrepancies(wr, ctx):
    """q = 64 with discrepancies of rank below m (sequences of a rank-5
    matrix, and one with zero columns): non-pivot columns before the m-th
    pivot, and orders with no pivot at all."""
    p = 1073741789
    rng = np.random.default_rng(11)
    m = n = 32
    U = rng.integers(0, p, size=(m, 5)).astype(object)
    V = rng.integers(0, p, size=(5, n)).astype(object)
    L = 40
    S = np.zeros((L, m, n), np.uint32)
    for k in range(L):
        Dk = np.diag(rng.integers(0, p, size=5).astype(object))
        S[k] = ((U.dot(Dk).dot(V)) % p).astype(np.uint32)
    S2 = S.copy()
    S2[:, :, 7] = 0
    S2[3] = 0
    for T in [S, S2]:
        M, deg = oracle.mbasis(T, p)
        P, dg = gpu_sigma(wr, ctx, T, p)
        assert np.array_equal(dg, deg)
        assert np.array_equal(P[: M.shape[0]], M[:, :n, :])


def test_sigma_basis_degenerate_sequences(wr, ctx):
    p = 1073741789
    for S in [np.zeros((20, 2, 2), np.uint32),
              np.concatenate([np.ones((1, 3, 3), np.uint32), np.zeros((30, 3, 3), np.uint32)]),
              np.tile(np.eye(2, dtype=np.uint32)[None], (25, 1, 1))]:
        M, deg = oracle.mbasis(S, p)
        P, dg = gpu_sigma(wr, ctx, S, p)
        n = S.shape[2]
        assert np.array_equal(dg, deg)
        assert np.array_equal(P[: M.shape[0]], M[:, :n, :])


# ------------------------------------------------------------------ det valuation (A9)

def test_det_valuation_parity(wr, ctx):
    p = 65521
    rng = np.random.default_rng(5)
    for t in range(20):
        n = int(rng.integers(1, 9))
        e = rng.integers(0, 3, size=n)
        U = rng.integers(0, p, size=(2, n, n))
        V = rng.integers(0, p, size=(2, n, n))
        U[0] = np.triu(U[0], 1) + np.eye(n, dtype=np.int64)
        V[0] = np.tril(V[0], -1) + np.eye(n, dtype=np.int64)
        Dg = np.zeros((int(e.max()) + 1, n, n), dtype=np.int64)
        for i in range(n):
            Dg[int(e[i]), i, i] = 1
        G = oracle.polymat_mul(oracle.polymat_mul(U, Dg, p), V, p).astype(np.uint32)
        # same precision on both sides (coefficients past the degree are 0);
        # the short one may legitimately not determine the valuation (-1)
        for T in [G.shape[0], 2 * G.shape[0] + 2 * n]:
            Gp = np.zeros((T, n, n), dtype=np.uint32)
            Gp[: G.shape[0]] = G
            v = wr.wr_det_valuation_device(ctx, to_dev(Gp), n, T, p)
            ref = oracle.load().or_det_valuation(oracle._p(Gp), n, T, p)
            assert v == ref
        assert v == oracle.det_valuation(G, p) == int(e.sum())


# ------------------------------------------------------------------ rank (A1-A9)

def gpu_rank(wr, ctx, A, p, m, n, seed, want=0, side=-1, symmetric=False):
    mat = load(wr, ctx, A)
    prm = wr.make_params(p, m, n, seed, side=side, want=want,
                         projection=wr.WR_PROJ_SYMMETRIC if symmetric else wr.WR_PROJ_GENERIC)
    res = wr.wr_rank(ctx, mat, prm)
    out = dict(rank=wr.wr_result_rank(res), **wr.wr_result_info(res))
    if want & wr.WR_WANT_SEQUENCE:
        out["S"] = wr.wr_result_sequence(res, m, n)
    if want & wr.WR_WANT_GENERATOR:
        out["F"], out["delta"] = wr.wr_result_generator(res, n)
    wr.wr_result_free(res)
    wr.wr_matrix_free(mat)
    return out


def test_rank_config0_scalar(wr, ctx):
    A = synth.config0()
    p = synth.PRIME_C0
    ref = oracle.rank_wiedemann(A, p, 1, 1, seed=synth.SEED_BASE)
    g = gpu_rank(wr, ctx, A, p, 1, 1, synth.SEED_BASE, want=3)
    assert g["rank"] == ref["rank"] == 1500
    assert (g["deg_det"], g["codeg"]) == (ref["deg_det"], ref["codeg"])
    assert np.array_equal(g["S"], ref["S"])
    assert np.array_equal(g["delta"], ref["delta"])
    assert np.array_equal(g["F"], ref["F"])


@pytest.mark.parametrize("m,n", [(2, 2), (4, 4), (8, 8), (3, 5)])
@pytest.mark.parametrize("p", PRIMES)
def test_rank_planted_block(wr, ctx, m, n, p):
    for t in range(3):
        rng = np.random.default_rng(t * 31 + m)
        R, C = int(rng.integers(50, 400)), int(rng.integers(50, 400))
        r = int(rng.integers(1, min(R, C)))
        A = synth.planted_sparse(R, C, r, row_len=int(rng.integers(2, 9)), seed=t + 100 * m)
        ref = oracle.rank_wiedemann(A, p, m, n, seed=t)
        g = gpu_rank(wr, ctx, A, p, m, n, t, want=3)
        assert g["rank"] == ref["rank"] == r
        assert (g["deg_det"], g["codeg"], g["sum_delta"]) == (ref["deg_det"], ref["codeg"], ref["sum_delta"])
        assert np.array_equal(g["F"], ref["F"])


def test_rank_edge_cases(wr, ctx):
    p = 65521
    Z = synth.csr_from_coo(5, 4, np.zeros(0), np.zeros(0), np.zeros(0))
    assert gpu_rank(wr, ctx, Z, p, 2, 2, 1)["rank"] == 0
    one = synth.dense_to_csr(np.array([[0, 1], [0, 0]]))
    assert gpu_rank(wr, ctx, one, p, 1, 1, 1)["rank"] == 1
    eye = synth.dense_to_csr(np.eye(40, dtype=np.int64))
    assert gpu_rank(wr, ctx, eye, p, 4, 4, 1)["rank"] == 40
    big = synth.dense_to_csr(np.array([[127, -127, 5], [-128 + 1, 3, 0]]))
    assert gpu_rank(wr, ctx, big, 2147483629, 1, 1, 3)["rank"] == oracle.rank_dense(big.to_dense(), 2147483629)
    # heavy rows and columns in a planted matrix
    H = heavy_matrix(900, 800, seed=3)
    ref = oracle.rank_sparse(H, 1073741789)
    assert gpu_rank(wr, ctx, H, 1073741789, 8, 8, 2)["rank"] == ref


def test_rank_chain_complex_pair(wr, ctx):
    d_n, d_n1 = synth.chain_pair(2500, seed=8, homology=3)
    p = 1073741783
    rn = gpu_rank(wr, ctx, d_n, p, 8, 8, 5)["rank"]
    rn1 = gpu_rank(wr, ctx, d_n1, p, 8, 8, 6)["rank"]
    assert rn == d_n.rank and rn1 == d_n1.rank
    assert rn + rn1 <= 2500


def test_errors_are_reported(wr, ctx):
    A = synth.random_sparse(10, 10, 2, seed=1)
    with pytest.raises(wr.WrError) as ei:
        gpu_rank(wr, ctx, A, 65520, 1, 1, 1)
    assert ei.value.status == wr.WR_ENOTPRIME
    bad = synth.CSR(2, 2, np.array([0, 1, 2]), np.array([0, 5], np.int32), np.array([1, 1], np.int32))
    with pytest.raises(wr.WrError) as ei:
        load(wr, ctx, bad)
    assert ei.value.status == wr.WR_EINVAL
    big = synth.CSR(1, 1, np.array([0, 1]), np.array([0], np.int32), np.array([40000], np.int32))
    with pytest.raises(wr.WrError) as ei:
        load(wr, ctx, big)
    assert ei.value.status == wr.WR_EOVERFLOW


@pytest.mark.parametrize("m,n,L,leaf", [(1, 1, 700, 64), (2, 3, 610, 64), (3, 2, 900, 200), (4, 4, 950, 128),
                                      (8, 8, 1300, 200), (8, 8, 700, 64), (5, 5, 390, 64), (1, 1, 9000, 512),
                                      (2, 2, 6100, 256), (16, 16, 500, 64), (32, 32, 200, 64), (24, 20, 200, 64)])
@pytest.mark.parametrize("p", [65521, 2147483629, 1073741789])
def test_pm_basis_matches_order_by_order(wr, ctx, m, n, L, leaf, p):
    """PM-Basis (recursive halving, NTT products over three FFT primes, CRT
    back to p) gives the order-by-order M-Basis bit for bit: the leaf size is
    forced small so that the sequence is split several times."""
    rng = np.random.default_rng(m * 7919 + n * 31 + L + leaf)
    S = rng.integers(0, p, size=(L, m, n)).astype(np.uint32)
    M, deg = oracle.mbasis(S, p)
    wr.wr_set_sigma_leaf(ctx, leaf)
    try:
        P, dg = gpu_sigma(wr, ctx, S, p)
    finally:
        wr.wr_set_sigma_leaf(ctx, 0)
    assert np.array_equal(dg, deg)
    D = M.shape[0] - 1
    assert np.array_equal(P[: D + 1], M[:, :n, :])
    assert not P[D + 1:].any()


def test_pm_basis_q64_matches_mbasis_on_the_device(wr, ctx):
    """q = m + n = 64 over 3,000 orders (products of more than 4,096 points:
    transforms in two shared-memory passes): PM-Basis with 256-order leaves
    gives the blocked M-Basis's basis bit for bit (both pinned against the
    oracle on smaller cases above)."""
    p, m, n, L = 2147483629, 32, 32, 3000
    rng = np.random.default_rng(64)
    S = rng.integers(0, p, size=(L, m, n)).astype(np.uint32)
    P0, d0 = gpu_sigma(wr, ctx, S, p)
    wr.wr_set_sigma_leaf(ctx, 256)
    try:
        P1, d1 = gpu_sigma(wr, ctx, S, p)
    finally:
        wr.wr_set_sigma_leaf(ctx, 0)
    assert np.array_equal(d0, d1)
    assert np.array_equal(P0, P1)


@pytest.mark.parametrize("m", [2, 4, 8])
def test_rank_with_pm_basis(wr, ctx, m):
    p = 1073741789
    for t in range(2):
        rng = np.random.default_rng(t * 13 + m)
        R, C = int(rng.integers(300, 700)), int(rng.integers(300, 700))
        r = int(rng.integers(100, min(R, C)))
        A = synth.planted_sparse(R, C, r, row_len=int(rng.integers(3, 8)), seed=t + 500 * m)
        ref = oracle.rank_wiedemann(A, p, m, m, seed=t)
        wr.wr_set_sigma_leaf(ctx, 64)
        try:
            g = gpu_rank(wr, ctx, A, p, m, m, t, want=3)
        finally:
            wr.wr_set_sigma_leaf(ctx, 0)
        assert g["rank"] == ref["rank"] == r
        assert (g["deg_det"], g["codeg"], g["sum_delta"]) == (ref["deg_det"], ref["codeg"], ref["sum_delta"])
        assert np.array_equal(g["F"], ref["F"])


# ------------------------------------------------------------------ full size: config 1

def _annihilates(S, F, delta, p, i):
    """sum_k S[i+k] F[k][:, j] = 0 mod p for each column j with i + delta_j < L.
    Exact in uint64: F's residues split into 15-bit halves and the sums over
    k taken in chunks of 512 coefficients, each reduced mod p (a chunk adds at
    most 512 n products below 2^46)."""
    L, m, n = S.shape
    for j in range(n):
        dj = int(delta[j])
        if i + dj >= L:
            continue
        tot = [0] * m
        for k0 in range(0, dj + 1, 512):
            k1 = min(dj + 1, k0 + 512)
            Sk = S[i + k0: i + k1].astype(np.uint64)            # (c, m, n)
            f = F[k0:k1, :, j].astype(np.uint64)                 # (c, n)
            lo, hi = f & 0x7FFF, f >> 15
            acc_lo = np.einsum("kar,kr->a", Sk, lo)
            acc_hi = np.einsum("kar,kr->a", Sk, hi)
            tot = [(t + int(a) + (int(b) % p) * (1 << 15)) % p for t, a, b in zip(tot, acc_lo, acc_hi)]
        if any(tot):
            return False
    return True


def _deep_step_check(wr, ctx, A, mat, st, seed, k):
    """Spot check of the graph-replayed loop at depth k (Section 2.5 step 2,
    two terms per application of the symmetric A~, Section 2.3).  The GPU runs
    k + 1 applications of the paired block [D1 X | D1 Y] and exports the block
    after k of them, [U_k | V_k] = [A~^k X | A~^k Y], and after k + 1.  From
    [U_k | V_k] the oracle recomputes S_2k = U_k^T V_k, the next block
    [A~ U_k | A~ V_k], S_2k+1 = U_k^T A~ V_k and S_2k+2 = (A~ U_k)^T (A~ V_k),
    which must equal the GPU's own terms and block bit for bit."""
    p, m, n, N = st.p, st.m, st.n, st.N
    L = 2 * k + 3
    prm = wr.make_params(p, m, n, seed)
    dS = torch.empty((L, m, n), dtype=torch.int32, device="cuda")
    snap = torch.empty((N, m + n), dtype=torch.int32, device="cuda")
    last = torch.empty((N, m + n), dtype=torch.int32, device="cuda")
    apps, paired = wr.wr_sequence_state_device(ctx, mat, prm, dS, L, k, snap, last)
    assert paired and apps == k + 1
    S = from_dev(dS)
    UV = from_dev(snap)
    if k == 0:
        assert np.array_equal(UV[:, :m], st.X) and np.array_equal(UV[:, m:], st.Y)
    assert np.array_equal(oracle.project(UV[:, :m], UV[:, m:], p), S[2 * k])
    nxt = oracle.blackbox_apply(A, p, st.side, st.D1, st.D2, UV)
    assert np.array_equal(from_dev(last), nxt)
    assert np.array_equal(oracle.project(UV[:, :m], np.ascontiguousarray(nxt[:, m:]), p), S[2 * k + 1])
    assert np.array_equal(oracle.project(np.ascontiguousarray(nxt[:, :m]), np.ascontiguousarray(nxt[:, m:]), p),
                          S[2 * k + 2])
    return S


@pytest.fixture(scope="module")
def config1():
    return synth.config1()


@pytest.fixture(scope="module")
def config2():
    return synth.config2()


def test_config1_full_size(wr, ctx, config1):
    """200,000 x 180,000, block 8 x 8, p = 1073741789: planted rank, the first
    terms against the oracle, the generator annihilates the sequence at
    sampled offsets, and one black-box application at full size."""
    A = config1
    p, m, n, seed = synth.PRIME_C1, 8, 8, synth.SEED_BASE + 1
    g = gpu_rank(wr, ctx, A, p, m, n, seed, want=3)
    assert g["rank"] == A.rank == 170000
    assert g["seq_len"] == 45002
    st = oracle.Setup(A, p, m, n, seed)
    S_ref = oracle.sequence(A, st, L=6)
    assert np.array_equal(g["S"][:6], S_ref)
    rng = np.random.default_rng(0)
    for i in [0, 1] + list(rng.integers(0, 22000, size=3)):
        assert _annihilates(g["S"], g["F"], g["delta"], p, int(i))
    mat = load(wr, ctx, A)
    v = rng.integers(0, p, size=(A.cols, n)).astype(np.uint32)
    dout = torch.empty((A.cols, n), dtype=torch.int32, device="cuda")
    wr.wr_blackbox_apply_device(ctx, mat, wr.make_params(p, 1, n, seed), to_dev(v), dout, n)
    ref = oracle.blackbox_apply(A, p, 0, st.D1, st.D2, v)
    assert np.array_equal(from_dev(dout), ref)
    wr.wr_matrix_free(mat)


@pytest.mark.parametrize("k", [0, 1000, 20001, 22499])
def test_config1_deep_steps(wr, ctx, config1, k):
    """Config 1 at depth k of its 22,501 applications (k = 22,499: the last
    graph group is partial), each step checked by the oracle from the GPU's
    own block; the terms S_2k .. S_2k+2 also sit in the full wr_rank sequence."""
    A = config1
    p, m, n, seed = synth.PRIME_C1, 8, 8, synth.SEED_BASE + 1
    st = oracle.Setup(A, p, m, n, seed)
    mat = load(wr, ctx, A)
    try:
        _deep_step_check(wr, ctx, A, mat, st, seed, k)
    finally:
        wr.wr_matrix_free(mat)


# ------------------------------------------------------------------ full size: config 2

def test_config2_full_size_spot_checks(wr, ctx, config2):
    """1,900,000 x 1,950,000, ~40.7M nnz, block 32 x 32, p = 2147483629 (rows
    side, N = 1.9M): one black-box application at full size checked on 64
    sampled output rows computed one by one, and the loop at depth 0 (the
    first three terms) and 4,100 (paired block of width 64, Gram projections
    on the tensor cores) checked step by step against the oracle."""
    A = config2
    p, m, n, seed = 2147483629, 32, 32, synth.SEED_BASE + 2
    st = oracle.Setup(A, p, m, n, seed)
    assert st.side == 1 and st.N == 1900000
    mat = load(wr, ctx, A)
    try:
        rng = np.random.default_rng(2)
        v = rng.integers(0, p, size=(st.N, n)).astype(np.uint32)
        dout = torch.empty((st.N, n), dtype=torch.int32, device="cuda")
        wr.wr_blackbox_apply_device(ctx, mat, wr.make_params(p, 1, n, seed), to_dev(v), dout, n)
        got = from_dev(dout)
        rows = np.sort(rng.choice(st.N, 64, replace=False))
        assert np.array_equal(got[rows], oracle.blackbox_apply_rows(A, p, st.side, st.D1, st.D2, v, rows))
        del got, v, dout
        # depth 0: the exported block is [X | Y] itself, so S_0, S_1, S_2 are
        # checked against the oracle's literal first terms
        _deep_step_check(wr, ctx, A, mat, st, seed, 0)
        _deep_step_check(wr, ctx, A, mat, st, seed, 4100)
    finally:
        wr.wr_matrix_free(mat)


def test_config2_rank(wr, ctx, config2):
    """The one-prime time to rank of config 2: wr_rank over all L = 118,752
    terms (59,376 applications of the width-64 paired block) and the M-Basis
    at q = 64 gives the planted rank 1,805,000; the generator annihilates the
    sequence at sampled offsets and the first terms equal the oracle's."""
    A = config2
    p, m, n, seed = 2147483629, 32, 32, synth.SEED_BASE + 2
    wr.wr_set_profiling(ctx, True)
    try:
        g = gpu_rank(wr, ctx, A, p, m, n, seed, want=3)
        tm = wr.wr_last_timings(ctx)
    finally:
        wr.wr_set_profiling(ctx, False)
    print("config 2 time to rank: %.1f s (sequence %.1f s, sigma-basis %.1f s, tail %.1f s)" % (
        tm["total_ms"] / 1e3, tm["sequence_ms"] / 1e3, tm["sigma_ms"] / 1e3, tm["sigma_tail_ms"] / 1e3))
    assert g["rank"] == A.rank == 1805000
    assert g["seq_len"] == 118752
    rng = np.random.default_rng(5)
    for i in [0] + list(rng.integers(0, 50000, size=2)):
        assert _annihilates(g["S"], g["F"], g["delta"], p, int(i))


def test_config2_rank_symmetric(wr, ctx, config2):
    """Config 2 with the symmetric projection of Section 2.3 (X = Y^T: two
    terms per application of the width-32 block): the planted rank 1,805,000, the generator annihilates the sequence
    at sampled offsets, and S_0 .. S_2 equal the oracle's literal loop."""
    A = config2
    p, m, n, seed = 2147483629, 32, 32, synth.SEED_BASE + 2
    g = gpu_rank(wr, ctx, A, p, m, n, seed, want=3, symmetric=True)
    assert g["rank"] == A.rank == 1805000
    assert g["seq_len"] == 118752
    rng = np.random.default_rng(6)
    for i in [0] + list(rng.integers(0, 50000, size=2)):
        assert _annihilates(g["S"], g["F"], g["delta"], p, int(i))
    st = oracle.Setup(A, p, m, n, seed=seed, symmetric=True)
    assert np.array_equal(g["S"][:3], oracle.sequence(A, st, 3))
