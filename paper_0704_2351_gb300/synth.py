"""Seeded synthetic inputs for the block Wiedemann rank path.

This module builds integer sparse matrices (CSR) and request traces.  It holds
none of the rank method's arithmetic (no modular reduction, no black box, no
generator): both the CUDA library's tests/bench and the CPU oracle draw their
inputs from here, and nothing else is shared between the two.

Workload shapes follow the paper's experiments (Section 3, Table "tab:res":
GL7d19 is 1,911,130 x 1,955,309 with 37,322,725 nonzeros, entries small
integers, most of them +-1).  The matrices of the paper are not available, so
every generator below plants a known rank by construction:

* base rows carry a unit pivot structure: base row i has +-1 in its own pivot
  column pi(i) and no entry in pi(j) for j < i.  Restricted to the pivot
  columns the base block is triangular with +-1 on the diagonal, hence
  nonsingular over every field;
* dependent rows are integer combinations of a few base rows, so they add no
  rank.

Hence rank_p(A) = number of base rows for every prime p, with no elimination
needed to know it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class CSR:
    """Integer sparse matrix in CSR form (rows sorted, columns sorted per row)."""
    rows: int
    cols: int
    rowptr: np.ndarray  # int64, rows+1
    colidx: np.ndarray  # int32, nnz
    vals: np.ndarray    # int32, nnz
    rank: Optional[int] = None  # planted rank, when known by construction

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def transpose(self) -> "CSR":
        order = np.lexsort((np.repeat(np.arange(self.rows, dtype=np.int64),
                                      np.diff(self.rowptr)), self.colidx))
        r = np.repeat(np.arange(self.rows, dtype=np.int32), np.diff(self.rowptr))[order]
        c = self.colidx[order]
        v = self.vals[order]
        ptr = np.zeros(self.cols + 1, dtype=np.int64)
        np.add.at(ptr, c.astype(np.int64) + 1, 1)
        np.cumsum(ptr, out=ptr)
        return CSR(self.cols, self.rows, ptr, r.astype(np.int32), v.astype(np.int32), self.rank)

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.rows, self.cols), dtype=np.int64)
        r = np.repeat(np.arange(self.rows), np.diff(self.rowptr))
        np.add.at(a, (r, self.colidx.astype(np.int64)), self.vals.astype(np.int64))
        return a


def csr_from_coo(rows: int, cols: int, r: np.ndarray, c: np.ndarray, v: np.ndarray,
                 rank: Optional[int] = None) -> CSR:
    """Sum duplicates, drop zeros, sort by (row, col)."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    key = r * cols + c
    order = np.argsort(key, kind="stable")
    key = key[order]
    v = v[order]
    uniq, start = np.unique(key, return_index=True)
    sums = np.add.reduceat(v, start) if len(v) else v
    keep = sums != 0
    uniq = uniq[keep]
    sums = sums[keep]
    rr = uniq // cols
    cc = uniq % cols
    ptr = np.zeros(rows + 1, dtype=np.int64)
    np.add.at(ptr, rr + 1, 1)
    np.cumsum(ptr, out=ptr)
    return CSR(rows, cols, ptr, cc.astype(np.int32), sums.astype(np.int32), rank)


def dense_to_csr(a: np.ndarray) -> CSR:
    a = np.asarray(a, dtype=np.int64)
    r, c = np.nonzero(a)
    return csr_from_coo(a.shape[0], a.shape[1], r, c, a[r, c])


# ---------------------------------------------------------------------------
# value and column distributions
# ---------------------------------------------------------------------------

def _values(rng: np.random.Generator, k: int, p_unit: float, vmax: int) -> np.ndarray:
    """+-1 with probability p_unit, else uniform in [-vmax, vmax] \\ {0}."""
    sign = rng.integers(0, 2, size=k) * 2 - 1
    big = rng.integers(1, vmax + 1, size=k) * (rng.integers(0, 2, size=k) * 2 - 1)
    unit = rng.random(k) < p_unit
    return np.where(unit, sign, big).astype(np.int64)


def zipf_column_weights(cols: int, alpha: float, rng: np.random.Generator) -> np.ndarray:
    """Power-law column degrees with exponent alpha: weight of the j-th most
    popular column is j^(-1/(alpha-1)); popularity ranks are shuffled over the
    column indices."""
    j = np.arange(1, cols + 1, dtype=np.float64)
    w = j ** (-1.0 / (alpha - 1.0))
    w /= w.sum()
    perm = rng.permutation(cols)
    out = np.empty(cols)
    out[perm] = w
    return out


class _ColumnSampler:
    def __init__(self, cols: int, weights: Optional[np.ndarray]):
        self.cols = cols
        if weights is None:
            self.cdf = None
        else:
            self.cdf = np.cumsum(weights)
            self.cdf /= self.cdf[-1]

    def draw(self, rng: np.random.Generator, k: int) -> np.ndarray:
        if self.cdf is None:
            return rng.integers(0, self.cols, size=k, dtype=np.int64)
        u = rng.random(k)
        return np.minimum(np.searchsorted(self.cdf, u, side="right"), self.cols - 1).astype(np.int64)


# ---------------------------------------------------------------------------
# planted-rank sparse matrices
# ---------------------------------------------------------------------------

def planted_sparse(rows: int, cols: int, rank: int, *, row_len, seed: int,
                   col_weights: Optional[np.ndarray] = None, p_unit: float = 0.95,
                   vmax: int = 3, dep_terms: int = 3, dep_coef: int = 2) -> CSR:
    """Random sparse integer matrix of exact rank `rank` over every prime field.

    row_len: int (every base row), or callable(rng, k) -> array of k lengths.
    col_weights: None for uniform columns, else a probability per column.
    Base rows: one +-1 pivot entry plus row_len-1 entries drawn from the column
    distribution, avoiding pivots of earlier base rows.  Dependent rows
    (rows - rank of them): sum of `dep_terms` distinct base rows with
    coefficients uniform in {+-1, ..., +-dep_coef}.  Rows are then shuffled.
    """
    assert 0 <= rank <= min(rows, cols)
    rng = np.random.default_rng(seed)
    sampler = _ColumnSampler(cols, col_weights)
    r = rank
    # Pivot columns.  With a column distribution, pivots are taken among the
    # less popular columns and ordered by popularity ascending, so that the
    # "avoid earlier pivots" rule only ever bars unpopular columns.
    if col_weights is None:
        piv = rng.permutation(cols)[:r].astype(np.int64)
    else:
        by_pop = np.argsort(col_weights, kind="stable")  # ascending popularity
        piv = by_pop[:r].astype(np.int64)
    piv_idx = np.full(cols, r, dtype=np.int64)  # r = "not a pivot"
    piv_idx[piv] = np.arange(r)

    if callable(row_len):
        lens = np.asarray(row_len(rng, r), dtype=np.int64)
    else:
        lens = np.full(r, int(row_len), dtype=np.int64)
    lens = np.clip(lens, 1, cols)

    out_r, out_c, out_v = [], [], []
    # pivot entries
    out_r.append(np.arange(r, dtype=np.int64))
    out_c.append(piv)
    out_v.append(rng.integers(0, 2, size=r).astype(np.int64) * 2 - 1)

    # other entries, drawn in blocks of rows with oversampling + rejection
    # row i may only use columns that are not pivots of rows <= i
    allowed = (cols - r) + (r - 1 - np.arange(r, dtype=np.int64))
    need = np.minimum(lens - 1, allowed)
    block = 65536
    for b0 in range(0, r, block):
        b1 = min(r, b0 + block)
        todo = np.arange(b0, b1, dtype=np.int64)
        todo = todo[need[todo] > 0]
        over = 3
        while len(todo):
            k_need = need[todo]
            # allowed fraction for row i: columns with piv_idx > i
            kk = int(k_need.max()) * over + 8
            cand = sampler.draw(rng, len(todo) * kk).reshape(len(todo), kk)
            ok = piv_idx[cand] > todo[:, None]
            # sequential draws without replacement: keep the first occurrence
            # of each column (in draw order) among the allowed ones
            order = np.argsort(cand, axis=1, kind="stable")
            srt = np.take_along_axis(cand, order, axis=1)
            first_sorted = np.ones_like(ok)
            first_sorted[:, 1:] = srt[:, 1:] != srt[:, :-1]
            first = np.empty_like(ok)
            np.put_along_axis(first, order, first_sorted, axis=1)
            valid = ok & first
            nvalid = valid.sum(axis=1)
            done = nvalid >= k_need
            if done.any():
                rows_d = todo[done]
                kd = k_need[done]
                valid_d = valid[done]
                rank_in_row = np.cumsum(valid_d, axis=1)
                sel = valid_d & (rank_in_row <= kd[:, None])
                picked = cand[done][sel]
                out_r.append(np.repeat(rows_d, kd))
                out_c.append(picked)
                out_v.append(_values(rng, len(picked), p_unit, vmax))
            todo = todo[~done]
            over *= 2

    br = np.concatenate(out_r)
    bc = np.concatenate(out_c)
    bv = np.concatenate(out_v)
    base = csr_from_coo(r, cols, br, bc, bv)

    # dependent rows
    nd = rows - r
    dr, dc, dv = [np.zeros(0, np.int64)] * 3
    if nd > 0 and r > 0:
        t = min(dep_terms, r)
        picks = np.stack([rng.choice(r, size=t, replace=False) for _ in range(nd)]) \
            if nd * t < 4096 else _distinct_rows(rng, nd, t, r)
        coef = rng.integers(1, dep_coef + 1, size=(nd, t)) * (rng.integers(0, 2, size=(nd, t)) * 2 - 1)
        rr, cc, vv = [], [], []
        for j in range(t):
            src = picks[:, j]
            ln = base.rowptr[src + 1] - base.rowptr[src]
            starts = np.repeat(base.rowptr[src], ln)
            within = np.arange(ln.sum()) - np.repeat(np.cumsum(ln) - ln, ln)
            idx = starts + within
            rr.append(np.repeat(np.arange(nd, dtype=np.int64), ln))
            cc.append(base.colidx[idx].astype(np.int64))
            vv.append(base.vals[idx].astype(np.int64) * np.repeat(coef[:, j], ln))
        dr, dc, dv = np.concatenate(rr) + r, np.concatenate(cc), np.concatenate(vv)
    elif nd > 0:
        dr = dc = dv = np.zeros(0, np.int64)

    allr = np.concatenate([np.repeat(np.arange(r, dtype=np.int64), np.diff(base.rowptr)), dr])
    allc = np.concatenate([base.colidx.astype(np.int64), dc])
    allv = np.concatenate([base.vals.astype(np.int64), dv])
    # hidden row shuffle
    perm = rng.permutation(rows)
    return csr_from_coo(rows, cols, perm[allr], allc, allv, rank=r)


def _distinct_rows(rng, nd, t, r):
    picks = rng.integers(0, r, size=(nd, t))
    for _ in range(64):
        bad = np.zeros(nd, dtype=bool)
        for a in range(t):
            for b in range(a + 1, t):
                bad |= picks[:, a] == picks[:, b]
        if not bad.any():
            return picks
        picks[bad] = rng.integers(0, r, size=(int(bad.sum()), t))
    raise RuntimeError("could not draw distinct base rows")


def random_sparse(rows: int, cols: int, density_per_row: int, *, seed: int, vmax: int = 3,
                  p_unit: float = 0.9) -> CSR:
    """Unstructured random sparse matrix (rank unknown a priori)."""
    rng = np.random.default_rng(seed)
    k = min(density_per_row, cols)
    r = np.repeat(np.arange(rows, dtype=np.int64), k)
    c = rng.integers(0, cols, size=rows * k)
    v = _values(rng, rows * k, p_unit, vmax)
    return csr_from_coo(rows, cols, r, c, v)


# ---------------------------------------------------------------------------
# chain complexes: d_n . d_{n+1} = 0 by construction
# ---------------------------------------------------------------------------

def chain_pair(c_n: int, *, seed: int, c_lo: Optional[int] = None, c_hi: Optional[int] = None,
               homology: int = 2, extra: int = 3):
    """Two boundary matrices d_n (c_{n-1} x c_n) and d_{n+1} (c_n x c_{n+1}) with
    d_n d_{n+1} = 0 over Z, as in a cellular chain complex (d o d = 0).

    C_n's coordinates are split in groups of t in [4, 8]; group g = a + b
    coordinates (plus, in `homology` groups, one spare coordinate).  Locally
    G_g = [-B_g | I_a] and H_g = [I_b ; B_g] with a small random integer B_g, so
    G_g H_g = 0 and ker G_g = im H_g.  Then d_n = F G P and d_{n+1} = P^T H J with
    a coordinate permutation P, F of full column rank and J of full row rank
    (unit pivots), so rank d_n = sum a, rank d_{n+1} = sum b and the homology
    dimension at C_n is the number of spare coordinates.
    Returns (d_n, d_{n+1}) as CSR with planted ranks.
    """
    rng = np.random.default_rng(seed)
    # groups
    sizes, spare = [], []
    tot = 0
    while tot < c_n:
        t = int(rng.integers(4, 9))
        t = min(t, c_n - tot)
        sizes.append(t)
        tot += t
    ng = len(sizes)
    spare_g = set(rng.choice(ng, size=min(homology, ng), replace=False).tolist()) if ng else set()
    Gr, Gc, Gv, Hr, Hc, Hv = [], [], [], [], [], []
    arow = 0  # rows of G (= sum a)
    bcol = 0  # cols of H (= sum b)
    off = 0
    for g, t in enumerate(sizes):
        s = 1 if (g in spare_g and t >= 3) else 0
        u = t - s
        if u < 2:
            off += t
            continue
        a = int(rng.integers(1, u))  # 1..u-1
        b = u - a
        B = rng.integers(-2, 3, size=(a, b))
        B[B == 0] = 1
        # coordinates of group: [off, off+b) -> first block (b coords), [off+b, off+u) -> a coords
        for i in range(a):
            for j in range(b):
                Gr.append(arow + i); Gc.append(off + j); Gv.append(-int(B[i, j]))
            Gr.append(arow + i); Gc.append(off + b + i); Gv.append(1)
        for j in range(b):
            Hr.append(off + j); Hc.append(bcol + j); Hv.append(1)
            for i in range(a):
                Hr.append(off + b + i); Hc.append(bcol + j); Hv.append(int(B[i, j]))
        arow += a
        bcol += b
        off += t
    G = csr_from_coo(arow, c_n, np.array(Gr), np.array(Gc), np.array(Gv))
    H = csr_from_coo(c_n, bcol, np.array(Hr), np.array(Hc), np.array(Hv))
    perm = rng.permutation(c_n)  # P: coordinate permutation
    c_lo = c_lo if c_lo is not None else max(arow, int(c_n * rng.uniform(0.5, 1.5)))
    c_hi = c_hi if c_hi is not None else max(bcol, int(c_n * rng.uniform(0.5, 1.5)))
    c_lo = max(c_lo, arow)
    c_hi = max(c_hi, bcol)
    F = _full_rank_factor(rng, c_lo, arow, extra, by_cols=True)   # c_lo x arow, full column rank
    J = _full_rank_factor(rng, c_hi, bcol, extra, by_cols=True).transpose()  # bcol x c_hi, full row rank
    # d_n = F G P ; (G P)[:, perm[j]] = G[:, j]
    GP = CSR(G.rows, G.cols, G.rowptr, perm[G.colidx].astype(np.int32), G.vals)
    GP = csr_from_coo(GP.rows, GP.cols, np.repeat(np.arange(GP.rows), np.diff(GP.rowptr)),
                      GP.colidx, GP.vals)
    d_n = spmul(F, GP)
    d_n.rank = arow
    # d_{n+1} = P^T H J ; (P^T H)[perm[j], :] = H[j, :]
    Hr_ = np.repeat(np.arange(H.rows), np.diff(H.rowptr))
    PH = csr_from_coo(H.rows, H.cols, perm[Hr_], H.colidx, H.vals)
    d_n1 = spmul(PH, J)
    d_n1.rank = bcol
    return d_n, d_n1


def _full_rank_factor(rng, rows, k, extra, by_cols=True) -> CSR:
    """rows x k integer matrix of full column rank k (k <= rows): column j has
    +-1 in its own pivot row, no entry in the pivot rows of earlier columns,
    plus `extra` random entries."""
    assert k <= rows
    piv = rng.permutation(rows)[:k]
    piv_idx = np.full(rows, k, dtype=np.int64)
    piv_idx[piv] = np.arange(k)
    rr = [piv.astype(np.int64)]
    cc = [np.arange(k, dtype=np.int64)]
    vv = [rng.integers(0, 2, size=k).astype(np.int64) * 2 - 1]
    if extra > 0 and k > 0:
        cand = rng.integers(0, rows, size=(k, extra * 4))
        ok = piv_idx[cand] > np.arange(k)[:, None]
        for j in range(extra):
            pass
        # take up to `extra` allowed candidates per column
        keys = np.where(ok, rng.random(ok.shape), 2.0)
        order = np.argsort(keys, axis=1)[:, :extra]
        chosen = np.take_along_axis(cand, order, axis=1)
        chosen_ok = np.take_along_axis(ok, order, axis=1)
        colj = np.repeat(np.arange(k), extra).reshape(k, extra)
        rr.append(chosen[chosen_ok])
        cc.append(colj[chosen_ok])
        vv.append(_values(rng, int(chosen_ok.sum()), 0.9, 2))
    return csr_from_coo(rows, k, np.concatenate(rr), np.concatenate(cc), np.concatenate(vv))


def spmul(a: CSR, b: CSR) -> CSR:
    """Exact integer sparse product a @ b (int64)."""
    assert a.cols == b.rows
    ar = np.repeat(np.arange(a.rows, dtype=np.int64), np.diff(a.rowptr))
    ac = a.colidx.astype(np.int64)
    av = a.vals.astype(np.int64)
    ln = b.rowptr[ac + 1] - b.rowptr[ac]
    starts = np.repeat(b.rowptr[ac], ln)
    within = np.arange(int(ln.sum())) - np.repeat(np.cumsum(ln) - ln, ln)
    idx = starts + within
    rr = np.repeat(ar, ln)
    cc = b.colidx[idx].astype(np.int64)
    vv = np.repeat(av, ln) * b.vals[idx].astype(np.int64)
    return csr_from_coo(a.rows, b.cols, rr, cc, vv)


# ---------------------------------------------------------------------------
# the workload configurations (sizes and distributions from the paper's table
# of GL7 boundary matrices; seeds are fixed per configuration)
# ---------------------------------------------------------------------------

SEED_BASE = 20070704

PRIME_C0 = 65521
PRIME_C1 = 1073741789
PRIME_C2 = 2147483629


def config0(seed: int = SEED_BASE + 0) -> CSR:
    """2,000 x 1,800, 12 nnz/row uniform columns, 95% +-1 else uniform in
    [-3,3]\\{0}; 1,500 base rows + 500 dependent rows -> rank 1,500."""
    return planted_sparse(2000, 1800, 1500, row_len=12, seed=seed, p_unit=0.95, vmax=3)


def config1(seed: int = SEED_BASE + 1, scale: float = 1.0) -> CSR:
    """200,000 x 180,000, 20 nnz/row, power-law column degrees (alpha 2.1);
    170,000 base + 30,000 dependent rows -> rank 170,000."""
    R = int(200000 * scale)
    C = int(180000 * scale)
    r = int(170000 * scale)
    rng = np.random.default_rng(seed ^ 0x5EED)
    w = zipf_column_weights(C, 2.1, rng)
    return planted_sparse(R, C, r, row_len=20, seed=seed, col_weights=w, p_unit=0.95, vmax=3)


def config2(seed: int = SEED_BASE + 2, scale: float = 1.0) -> CSR:
    """1,900,000 x 1,950,000, Poisson(19.5) row lengths, uniform columns, 97%
    +-1 else uniform in [-4,4]\\{0}; 5% rank deficit -> rank 1,805,000."""
    R = int(1900000 * scale)
    C = int(1950000 * scale)
    r = int(round(R * 0.95))

    def lens(rng, k):
        return np.maximum(1, rng.poisson(19.5, size=k))
    return planted_sparse(R, C, r, row_len=lens, seed=seed, p_unit=0.97, vmax=4)


def log_uniform_int(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size)).astype(np.int64)


def config3_pairs(npairs: int = 64, seed: int = SEED_BASE + 3, lo: int = 5000, hi: int = 300000):
    """Chain-complex pairs with row counts log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(npairs):
        c_n = int(log_uniform_int(rng, lo, hi))
        out.append(chain_pair(c_n, seed=seed * 1000 + k, homology=int(rng.integers(0, 6))))
    return out


def config4_trace(nreq: int = 1000, rate: float = 200.0, seed: int = SEED_BASE + 4,
                  lo: int = 1000, hi: int = 500000):
    """Poisson arrival trace of rank queries: list of dicts with arrival time,
    matrix shape, row length range, planted rank and seed (matrices are built
    lazily with planted_sparse)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    reqs = []
    for i in range(nreq):
        R = int(log_uniform_int(rng, lo, hi))
        C = max(1, int(math.ceil(R * rng.uniform(0.85, 1.0))))
        reqs.append(dict(t=float(t[i]), rows=R, cols=C, rank=int(0.95 * min(R, C)),
                         seed=int(seed * 100000 + i), prime_slot=int(rng.integers(0, 4))))
    return reqs


def config4_matrix(req) -> CSR:
    def lens(rng, k):
        return rng.integers(10, 21, size=k)
    return planted_sparse(req["rows"], req["cols"], req["rank"], row_len=lens, seed=req["seed"])
