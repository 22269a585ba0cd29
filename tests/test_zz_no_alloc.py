"""The allocation-free black-box call gives the same result as the ordinary
one.

wr_blackbox_apply_device_noalloc serves callers that must not allocate device
memory while they run (code inside another program's fixed memory arena,
latency-critical loops where cudaMalloc/cudaFree would stall the device).  It
keeps its temporaries in one fixed per-device array, so two calls in a row
also check that nothing left there by the first call leaks into the second.
This file is collected last on purpose.
"""
import numpy as np
import pytest

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


def _matrix(seed):
    """Sparse matrix with a few rows and columns long enough to be cut into
    segments, so both passes use the split-row accumulators."""
    rng = np.random.default_rng(seed)
    R, C = 3000, 2600
    base = synth.random_sparse(R, C, 6, seed=seed)
    r = [np.repeat(np.arange(R), np.diff(base.rowptr))]
    c = [base.colidx.astype(np.int64)]
    v = [base.vals.astype(np.int64)]
    for _ in range(4):
        row = int(rng.integers(0, R))
        cols = rng.choice(C, size=900, replace=False)
        r.append(np.full(900, row)); c.append(cols); v.append(rng.choice([-2, -1, 1, 3], size=900))
        col = int(rng.integers(0, C))
        rows = rng.choice(R, size=1100, replace=False)
        r.append(rows); c.append(np.full(1100, col)); v.append(rng.choice([-1, 1, 2], size=1100))
    return synth.csr_from_coo(R, C, np.concatenate(r), np.concatenate(c), np.concatenate(v))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


@pytest.mark.parametrize("width,side,p", [(8, 0, 1073741789), (3, 1, 2147483629), (32, 0, 65521)])
def test_noalloc_matches_blackbox_apply_twice(wr, ctx, width, side, p):
    A = _matrix(width + side)
    mat = wr.wr_matrix_load_csr(ctx, A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    N = A.cols if side == 0 else A.rows
    rng = np.random.default_rng(7)
    for call in range(2):
        prm = wr.make_params(p, 1, width, seed=100 + call, side=side)
        v = _dev(rng.integers(0, p, size=(N, width)))
        ref = torch.empty((N, width), dtype=torch.int32, device="cuda")
        out = torch.full((N, width), -1, dtype=torch.int32, device="cuda")
        wr.wr_blackbox_apply_device(ctx, mat, prm, v, ref, width)
        wr.wr_blackbox_apply_device_noalloc(ctx, mat, prm, v, out, width)
        assert torch.equal(out, ref), "call %d differs" % call
    wr.wr_matrix_free(mat)


def test_noalloc_rejects_requests_beyond_its_scratch(wr, ctx):
    R = C = 300000  # 4 * 32 * 600k bytes of blocks alone exceed 32 MiB
    rows = np.arange(R)
    A = synth.csr_from_coo(R, C, rows, rows, np.ones(R, dtype=np.int64))
    mat = wr.wr_matrix_load_csr(ctx, A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    v = torch.zeros((C, 32), dtype=torch.int32, device="cuda")
    out = torch.zeros((C, 32), dtype=torch.int32, device="cuda")
    with pytest.raises(wr.WrError) as ei:
        wr.wr_blackbox_apply_device_noalloc(ctx, mat, wr.make_params(65521, 1, 32, 1), v, out, 32)
    assert ei.value.status == wr.WR_EINVAL
    assert "bytes of scratch" in ei.value.message
    wr.wr_matrix_free(mat)
