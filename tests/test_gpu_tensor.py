"""The tensor-core Gram projection (tcgen05, bf16 digit products) against the
oracle: the probe's raw MMA layout against an exact integer product, the
Gram product G = sum_r w_r L_r^T R_r mod p against the oracle's projection on
shapes, sizes and residue extremes, and whole sequences with the tensor-core
path forced on and off against the oracle's literal loop.  Integer work:
every comparison is exact."""
import numpy as np
import pytest

import oracle
from paper_0704_2351_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_probe_layout_is_the_exact_product(wr, ctx):
    """One block, one chain of four MMAs (K = 64): the fp32 accumulator equals
    the integer product of the probe's tiles, entry by entry (checks the
    swizzled operand layout, the descriptors and the TMEM lane/column map)."""
    out = torch.zeros((128, 256), dtype=torch.float32, device="cuda")
    wr.wr_probe_mma(ctx, 1, 1, out)
    r = np.arange(128)[:, None]
    c = np.arange(256)[:, None]
    k = np.arange(64)[None, :]
    a = (r * 7 + k * 3) % 17 - 8
    b = (c * 5 + k * 11) % 13 - 6
    ref = a @ b.T
    assert np.array_equal(out.cpu().numpy().astype(np.int64), ref)
    out.zero_()
    wr.wr_probe_mma(ctx, 3, 2, out)  # accumulation over chains
    assert np.array_equal(out.cpu().numpy().astype(np.int64), 3 * ref)


def gram_ref(t, w, m, n, yoff, p):
    """G = sum_r w_r t[r][:m]^T t[r][yoff:yoff+n] mod p with the oracle's projection."""
    L = t[:, :m].astype(np.uint64)
    Lw = (L * w.astype(np.uint64)[:, None]) % np.uint64(p)
    return oracle.project(Lw.astype(np.uint32), np.ascontiguousarray(t[:, yoff:yoff + n]), p)


@pytest.mark.parametrize("m,n,tstride,yoff", [(32, 32, 64, 32), (32, 32, 32, 0), (16, 16, 32, 16), (16, 16, 16, 0),
                                              (8, 8, 16, 8), (8, 8, 8, 0), (5, 3, 8, 4), (32, 7, 32, 8),
                                              (12, 16, 32, 16)])
@pytest.mark.parametrize("N", [1, 63, 64, 65, 511, 513, 4097, 70001])
def test_gram_tensor_and_integer_paths_equal_the_oracle(wr, ctx, m, n, tstride, yoff, N):
    p = 2147483629
    rng = np.random.default_rng(N * 31 + m * 7 + n)
    t = rng.integers(0, p, size=(N, tstride), dtype=np.int64).astype(np.uint32)
    w = rng.integers(1, p, size=N, dtype=np.int64).astype(np.uint32)
    ref = gram_ref(t, w, m, n, yoff, p)
    G = torch.empty((m, n), dtype=torch.int32, device="cuda")
    try:
        for mode in [1, 0]:
            wr.wr_set_tensor_projection(ctx, mode)
            wr.wr_gram_device(ctx, p, N, m, n, to_dev(t), tstride, yoff, to_dev(w), G)
            assert np.array_equal(from_dev(G), ref), "mode %d" % mode
    finally:
        wr.wr_set_tensor_projection(ctx, -1)


@pytest.mark.parametrize("p", [65521, 1073741789, 2147483629, 2147483647])
def test_gram_residue_extremes(wr, ctx, p):
    """All entries p - 1 (the largest top digit, 128, at p near 2^31), zeros, ones,
    and a mix, over 3,000 rows (several drains of the fp32 accumulator)."""
    N, m, n = 3000, 32, 32
    rng = np.random.default_rng(p % 1000)
    cases = [np.full((N, 64), p - 1, dtype=np.uint32), np.zeros((N, 64), dtype=np.uint32),
             np.ones((N, 64), dtype=np.uint32),
             rng.choice(np.array([0, 1, p - 1, p // 2, (p + 1) // 2, 255, 256, 0x808080 % p], dtype=np.uint32),
                        size=(N, 64))]
    G = torch.empty((m, n), dtype=torch.int32, device="cuda")
    try:
        wr.wr_set_tensor_projection(ctx, 1)
        for t in cases:
            for w in [np.full(N, p - 1, dtype=np.uint32), rng.integers(1, p, size=N).astype(np.uint32)]:
                wr.wr_gram_device(ctx, p, N, m, n, to_dev(t), 64, 32, to_dev(w), G)
                assert np.array_equal(from_dev(G), gram_ref(t, w, m, n, 32, p))
    finally:
        wr.wr_set_tensor_projection(ctx, -1)


def test_gram_rejects_bad_shapes(wr, ctx):
    G = torch.empty((4, 4), dtype=torch.int32, device="cuda")
    t = torch.zeros((10, 8), dtype=torch.int32, device="cuda")
    w = torch.ones(10, dtype=torch.int32, device="cuda")
    for args in [(10, 4, 4, t, 6, 0), (10, 4, 4, t, 8, 2), (10, 33, 4, t, 8, 0), (10, 4, 4, t, 4, 4)]:
        with pytest.raises(wr.WrError):
            wr.wr_gram_device(ctx, 65521, *args[:4], args[4], args[5], w, G)


def heavy(R, C, seed):
    rng = np.random.default_rng(seed)
    base = synth.random_sparse(R, C, 6, seed=seed)
    r = [np.repeat(np.arange(R), np.diff(base.rowptr))]
    c = [base.colidx.astype(np.int64)]
    v = [base.vals.astype(np.int64)]
    for _ in range(2):  # a row and a column longer than one segment
        row = int(rng.integers(0, R))
        cols = rng.choice(C, size=min(600, C), replace=False)
        r.append(np.full(len(cols), row)); c.append(cols); v.append(rng.choice([-1, 1, 2], size=len(cols)))
        col = int(rng.integers(0, C))
        rows = rng.choice(R, size=min(600, R), replace=False)
        r.append(rows); c.append(np.full(len(rows), col)); v.append(rng.choice([-1, 1, 3], size=len(rows)))
    return synth.csr_from_coo(R, C, np.concatenate(r), np.concatenate(c), np.concatenate(v))


@pytest.mark.parametrize("n,sym,side,L", [(32, False, 0, 65), (32, False, 1, 64), (32, True, 0, 41), (16, False, 1, 57),
                                          (16, True, 1, 30), (8, False, 0, 49), (4, False, 1, 33), (20, False, 0, 37)])
@pytest.mark.parametrize("p", [65521, 2147483629])
def test_sequence_with_tensor_projection(wr, ctx, n, sym, side, L, p):
    """Whole sequences (paired generic at widths up to 64, and symmetric) with
    the Gram projections on the tensor cores and on the integer path, against
    the oracle's literal loop."""
    A = heavy(760, 700, seed=n * 13 + side + (5 if sym else 0))
    st = oracle.Setup(A, p, n, n, seed=70 + n, side=side, symmetric=sym)
    S_ref = oracle.sequence(A, st, L)
    mat = wr.wr_matrix_load_csr(ctx, A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    prm = wr.make_params(p, n, n, 70 + n, side=side, projection=wr.WR_PROJ_SYMMETRIC if sym else wr.WR_PROJ_GENERIC)
    dS = torch.empty((L, n, n), dtype=torch.int32, device="cuda")
    try:
        for mode in [1, 0, -1]:
            wr.wr_set_tensor_projection(ctx, mode)
            wr.wr_sequence_device(ctx, mat, prm, dS, L)
            assert np.array_equal(from_dev(dS), S_ref), "mode %d" % mode
    finally:
        wr.wr_set_tensor_projection(ctx, -1)
        wr.wr_matrix_free(mat)
