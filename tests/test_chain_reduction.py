"""Read-time host passes, no device needed.  Chain reduction (Section 2.6.4,
wr_chain_reduce_csr) checked against the oracle's Gaussian elimination.  For every matrix and prime,
rank_p(A) = rank_offset + rank_p(reduced), the reduced matrix keeps no unit
singleton row or column and no empty one, and the remaining rows and columns
keep their input order.  Locality order (wr_locality_order_csr): a
simultaneous renumbering of rows and columns by decreasing entry count."""
import numpy as np
import pytest

import oracle
from paper_0704_2351_gb300 import synth

PRIMES = [3, 5, 65521, 1073741789]


@pytest.fixture(scope="module")
def wr():
    from paper_0704_2351_gb300 import _build
    _build.build()
    from paper_0704_2351_gb300 import wr as w
    return w


def _reduce(wr, A, maps=False):
    r, c, rp, ci, va, rof, cof, off = wr.wr_chain_reduce_csr(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    R = synth.CSR(r, c, rp, ci, va)
    return (R, off, rof, cof) if maps else (R, off)


def _check_fixed_point(R):
    d = R.to_dense()
    for i in range(R.rows):
        nz = np.nonzero(d[i])[0]
        assert len(nz) >= 1, "empty row left"
        assert not (len(nz) == 1 and abs(d[i, nz[0]]) == 1), "unit singleton row left"
    for j in range(R.cols):
        nz = np.nonzero(d[:, j])[0]
        assert len(nz) >= 1, "empty column left"
        assert not (len(nz) == 1 and abs(d[nz[0], j]) == 1), "unit singleton column left"


def _mats():
    out = []
    for s in range(6):
        out.append(synth.planted_sparse(90 + 13 * s, 80 + 7 * s, 50 + 5 * s, row_len=3 + s % 3, seed=s))
        out.append(synth.random_sparse(70 + 9 * s, 75, 2 + s % 3, seed=100 + s, vmax=3, p_unit=0.6))
    d_n, d_n1 = synth.chain_pair(300, seed=7, homology=3)
    out += [d_n, d_n1]
    return out


def test_rank_is_offset_plus_reduced_rank(wr):
    for A in _mats():
        R, off = _reduce(wr, A)
        assert 0 <= off <= min(A.rows, A.cols)
        assert R.rows + off <= A.rows and R.cols + off <= A.cols
        for p in PRIMES:
            assert oracle.rank_dense(A.to_dense(), p) == off + oracle.rank_dense(R.to_dense(), p), p
        _check_fixed_point(R)


def test_entries_that_vanish_mod_p_are_never_pivots(wr):
    # a single entry 3 (zero mod 3) and a single entry 2: neither is a unit,
    # so nothing is taken (the rank is 1 mod 3 and 2 mod 5)
    A = synth.dense_to_csr(np.array([[3, 0], [0, 2]]))
    R, off = _reduce(wr, A)
    assert off == 0 and (R.rows, R.cols) == (2, 2)
    assert oracle.rank_dense(A.to_dense(), 3) == 1 and oracle.rank_dense(A.to_dense(), 5) == 2


def test_cascade_and_edge_cases(wr):
    # unit bidiagonal: one singleton starts a cascade through the whole matrix
    n = 40
    a = np.eye(n, dtype=np.int64) + np.diag(-np.ones(n - 1, dtype=np.int64), 1)
    R, off = _reduce(wr, synth.dense_to_csr(a))
    assert off == n and R.rows == 0 and R.cols == 0
    # empty matrix and all-zero rows/columns
    Z = synth.csr_from_coo(5, 4, np.zeros(0), np.zeros(0), np.zeros(0))
    R, off = _reduce(wr, Z)
    assert off == 0 and R.rows == 0 and R.cols == 0
    E = synth.csr_from_coo(0, 0, np.zeros(0), np.zeros(0), np.zeros(0))
    R, off = _reduce(wr, E)
    assert off == 0 and R.rows == 0
    # a dense block survives untouched, its empty border goes
    b = np.zeros((6, 7), dtype=np.int64)
    b[1:4, 2:5] = [[1, 2, 1], [2, 1, 1], [1, 1, 2]]
    R, off = _reduce(wr, synth.dense_to_csr(b))
    assert off == 0 and np.array_equal(R.to_dense(), b[1:4, 2:5])


def test_reduced_matrix_is_an_ordered_submatrix(wr):
    for A in _mats():
        R, off, rof, cof = _reduce(wr, A, maps=True)
        assert np.all(np.diff(rof) > 0) and np.all(np.diff(cof) > 0)
        d = A.to_dense()
        assert np.array_equal(R.to_dense(), d[np.ix_(rof, cof)])
        # what was removed: each pivot row/column pair plus empty lines; the
        # kept block meets no removed pivot (a unit singleton's row or column)
        assert R.rows + off <= A.rows and R.cols + off <= A.cols


def test_malformed_csr_is_rejected(wr):
    with pytest.raises(wr.WrError):
        wr.wr_chain_reduce_csr(2, 2, np.array([0, 1, 1]), np.array([5], dtype=np.int32),
                               np.array([1], dtype=np.int32))
    with pytest.raises(wr.WrError):
        wr.wr_chain_reduce_csr(2, 2, np.array([0, 2, 1]), np.array([0, 1], dtype=np.int32),
                               np.array([1, 1], dtype=np.int32))


def test_locality_order_is_a_degree_sorted_permutation(wr):
    for A in _mats() + [synth.config1(scale=0.01)]:
        rp, ci, va, rof, cof = wr.wr_locality_order_csr(A.rows, A.cols, A.rowptr, A.colidx, A.vals)
        assert sorted(rof) == list(range(A.rows)) and sorted(cof) == list(range(A.cols))
        B = synth.CSR(A.rows, A.cols, rp, ci, va)
        assert np.array_equal(B.to_dense(), A.to_dense()[np.ix_(rof, cof)])
        rlen = np.diff(A.rowptr)[rof]
        clen = np.bincount(A.colidx, minlength=A.cols)[cof]
        for lens, idx in [(rlen, rof), (clen, cof)]:
            assert np.all(np.diff(lens) <= 0), "not by decreasing entry count"
            ties = np.diff(lens) == 0
            assert np.all(np.diff(idx)[ties] > 0), "ties not by index"
        # columns sorted within each row
        for i in range(B.rows):
            assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)
        assert oracle.rank_dense(B.to_dense(), 65521) == oracle.rank_dense(A.to_dense(), 65521)


# ---------------------------------------------------------------------------
# along a complex: reductions propagate from one matrix to its neighbours
# ---------------------------------------------------------------------------

def _csr_tuple(A):
    return (A.rows, A.cols, A.rowptr, A.colidx, A.vals)


def _reduced(t):
    r, c, rp, ci, va, rof, cof, off = t
    return synth.CSR(r, c, rp, ci, va), rof, cof, off


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_complex_reduction_keeps_every_rank(wr, seed):
    d_n, d_n1 = synth.chain_pair(260 + 40 * seed, seed=seed, homology=seed % 3)
    out = wr.wr_chain_reduce_complex([_csr_tuple(d_n), _csr_tuple(d_n1)])
    for A, t in zip([d_n, d_n1], out):
        R, rof, cof, off = _reduced(t)
        assert np.array_equal(R.to_dense(), A.to_dense()[np.ix_(rof, cof)])
        for p in [3, 65521, 1073741789]:
            assert oracle.rank_dense(A.to_dense(), p) == off + oracle.rank_dense(R.to_dense(), p), p
        assert off + oracle.rank_dense(R.to_dense(), 1073741789) == A.rank
    # the reduced pair is still a complex over the same cells: d_n keeps as
    # columns exactly the cells d_n+1 keeps as rows, and the product is zero
    R_n, rof_n, cof_n, _ = _reduced(out[0])
    R_n1, rof_n1, cof_n1, off_n1 = _reduced(out[1])
    assert R_n.cols == R_n1.rows and np.array_equal(cof_n, rof_n1)
    assert not (R_n.to_dense() @ R_n1.to_dense()).any()
    # so the reduction runs again on its own output, and finds nothing more
    again = wr.wr_chain_reduce_complex([_csr_tuple(R_n), _csr_tuple(R_n1)])
    for R, t in zip([R_n, R_n1], again):
        R2, _, _, off2 = _reduced(t)
        assert off2 == 0 and (R2.rows, R2.cols) == (R.rows, R.cols)
        assert np.array_equal(R2.to_dense(), R.to_dense())


def test_complex_reduction_propagates_beyond_the_single_matrix_pass(wr):
    """A small complex where the neighbour's rule frees new singletons: the
    boundary of a filled square (2 triangles) -- d1: edges -> vertices,
    d2: faces -> edges.  Each matrix alone has no unit singleton row or
    column beyond what the pair unlocks."""
    # vertices 0..3, edges (0,1),(1,2),(2,3),(3,0),(0,2), faces (0,1,2),(0,2,3)
    e = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)]
    d1 = np.zeros((4, 5), dtype=np.int64)
    for j, (a, b) in enumerate(e):
        d1[a, j], d1[b, j] = -1, 1
    # faces (0,1,2) = e01 + e12 - e02 and (0,2,3) = e02 + e23 + e30
    d2 = np.array([[1, 0], [1, 0], [0, 1], [0, 1], [-1, 1]], dtype=np.int64)
    assert not (d1 @ d2).any()
    A1, A2 = synth.dense_to_csr(d1), synth.dense_to_csr(d2)
    single = [wr.wr_chain_reduce_csr(*_csr_tuple(A))[-1] for A in (A1, A2)]
    out = wr.wr_chain_reduce_complex([_csr_tuple(A1), _csr_tuple(A2)])
    offs = [t[-1] for t in out]
    # alone, d1 has no unit singleton line and d2 two; along the complex the
    # pivots of d2 free d1's rows: the contractible square reduces to nothing
    assert single == [0, 2] and offs == [3, 2]
    assert all(t[0] == 0 or t[1] == 0 for t in out)
    for A, t in zip([A1, A2], out):
        R, _, _, off = _reduced(t)
        assert oracle.rank_dense(A.to_dense(), 65521) == off + oracle.rank_dense(R.to_dense(), 65521)
    # the square is contractible: rank d1 = 3, rank d2 = 2
    assert oracle.rank_dense(d1, 65521) == 3 and oracle.rank_dense(d2, 65521) == 2


def test_complex_of_one_matrix_is_the_single_reduction(wr):
    for A in _mats():
        a = wr.wr_chain_reduce_csr(*_csr_tuple(A))
        b = wr.wr_chain_reduce_complex([_csr_tuple(A)])[0]
        assert a[0] == b[0] and a[1] == b[1] and a[-1] == b[-1]
        R1, R2 = synth.CSR(a[0], a[1], a[2], a[3], a[4]), synth.CSR(b[0], b[1], b[2], b[3], b[4])
        assert oracle.rank_dense(R1.to_dense(), 65521) == oracle.rank_dense(R2.to_dense(), 65521)


def test_complex_reduction_rejects_a_non_complex(wr):
    A = synth.dense_to_csr(np.array([[1, 1], [0, 1]]))
    B = synth.dense_to_csr(np.array([[1, 0], [0, 1]]))
    with pytest.raises(wr.WrError):
        wr.wr_chain_reduce_complex([_csr_tuple(A), _csr_tuple(B)])
    C = synth.dense_to_csr(np.array([[1, 0, 0]]))
    with pytest.raises(wr.WrError):  # 1 x 3 then 2 x 2: sizes do not chain
        wr.wr_chain_reduce_complex([_csr_tuple(C), _csr_tuple(B)])
