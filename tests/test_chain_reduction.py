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
