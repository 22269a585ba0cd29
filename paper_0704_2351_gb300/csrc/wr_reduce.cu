// Read-time passes on the host: the chain reduction (Section 2.6.4 "Chain
// Reductions") and the locality order.
//
// Chain reduction.
// A row whose only nonzero entry is lambda at column b (a free face when
// lambda = +-1) is removed together with column b: Gaussian elimination on
// that pivot changes nothing else (the paper's Eq. for the reduced
// differential with [v : a] = 0 on every other column), so
// rank(A) = 1 + rank(A without the row and the column).  The same holds for a
// column with a single entry (the transposed case).  Removals cascade: taking
// column b away can leave other rows with a single entry.  Empty rows and
// columns are dropped as well (they add nothing to the rank).
//
// Only unit pivots (lambda = +-1) are taken: they are units modulo every
// prime, so one reduced matrix serves all primes (rank over Q as the maximum
// over several p), and an entry that vanishes modulo some p is never taken
// for a pivot.  Entries stored as 0 are treated as absent.
//
// Host code, O(nnz) after the transposed index is built; it runs where the
// paper ran it, while the matrix is read.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "wr_internal.cuh"

namespace wr {

wr_status chain_reduce_host(int64_t rows, int64_t cols, const int64_t *rowptr, const int32_t *colidx,
                            const int32_t *vals, ReducedCsr &out) {
    if (rows < 0 || cols < 0) return fail(WR_EINVAL, "negative size");
    if (rows >= (int64_t(1) << 31) || cols >= (int64_t(1) << 31))
        return fail(WR_EOVERFLOW, "rows and cols must be < 2^31");
    if (!rowptr) return fail(WR_EINVAL, "null row pointer array");
    if (rowptr[0] != 0) return fail(WR_EINVAL, "rowptr[0] must be 0");
    for (int64_t i = 0; i < rows; i++)
        if (rowptr[i + 1] < rowptr[i]) return fail(WR_EINVAL, "rowptr must be nondecreasing");
    const int64_t nnz = rowptr[rows];
    if (nnz > 0 && (!colidx || !vals)) return fail(WR_EINVAL, "null column or value array");
    for (int64_t e = 0; e < nnz; e++)
        if (colidx[e] < 0 || colidx[e] >= cols) return fail(WR_EINVAL, "column index out of range");

    // entries per row and per column (nonzero values only), and the
    // transposed index: for column j, the entries e of A in it
    std::vector<int32_t> rcnt(rows, 0), ccnt(cols, 0);
    std::vector<int64_t> cptr(cols + 1, 0);
    for (int64_t i = 0; i < rows; i++)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++)
            if (vals[e] != 0) {
                rcnt[i]++;
                cptr[colidx[e] + 1]++;
            }
    for (int64_t j = 0; j < cols; j++) {
        ccnt[j] = (int32_t)cptr[j + 1];
        cptr[j + 1] += cptr[j];
    }
    std::vector<int32_t> crow(cptr[cols]);  // row of each entry, by column
    {
        std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
        for (int64_t i = 0; i < rows; i++)
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++)
                if (vals[e] != 0) crow[fill[colidx[e]]++] = (int32_t)i;
    }
    std::vector<char> rdead(rows, 0), cdead(cols, 0);
    std::deque<int64_t> rq, cq;
    for (int64_t i = 0; i < rows; i++)
        if (rcnt[i] == 1) rq.push_back(i);
    for (int64_t j = 0; j < cols; j++)
        if (ccnt[j] == 1) cq.push_back(j);
    int64_t pivots = 0;
    // value of A[i][j] among the live entries of row i (0 if none)
    auto row_single = [&](int64_t i, int64_t &jout) -> int32_t {
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++)
            if (vals[e] != 0 && !cdead[colidx[e]]) {
                jout = colidx[e];
                return vals[e];
            }
        return 0;
    };
    auto entry = [&](int64_t i, int64_t j) -> int32_t {
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++)
            if (colidx[e] == j && vals[e] != 0) return vals[e];
        return 0;
    };
    // remove row i and column j (pivot), updating the counts of the rows of
    // column j and the columns of row i
    auto take = [&](int64_t i, int64_t j) {
        rdead[i] = 1;
        cdead[j] = 1;
        pivots++;
        for (int64_t e = cptr[j]; e < cptr[j + 1]; e++) {
            const int64_t k = crow[e];
            if (!rdead[k] && --rcnt[k] == 1) rq.push_back(k);
        }
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            const int64_t c = colidx[e];
            if (vals[e] != 0 && !cdead[c] && --ccnt[c] == 1) cq.push_back(c);
        }
    };
    while (!rq.empty() || !cq.empty()) {
        while (!rq.empty()) {
            const int64_t i = rq.front();
            rq.pop_front();
            if (rdead[i] || rcnt[i] != 1) continue;
            int64_t j = -1;
            const int32_t v = row_single(i, j);
            if (v == 1 || v == -1) take(i, j);
        }
        while (!cq.empty()) {
            const int64_t j = cq.front();
            cq.pop_front();
            if (cdead[j] || ccnt[j] != 1) continue;
            int64_t i = -1;
            for (int64_t e = cptr[j]; e < cptr[j + 1]; e++)
                if (!rdead[crow[e]]) {
                    i = crow[e];
                    break;
                }
            if (i < 0) continue;
            const int32_t v = entry(i, j);
            if (v == 1 || v == -1) take(i, j);
        }
    }
    // compact: live rows and columns that still hold an entry
    std::vector<int32_t> cnew(cols, -1);
    int64_t nc = 0;
    for (int64_t j = 0; j < cols; j++)
        if (!cdead[j] && ccnt[j] > 0) cnew[j] = (int32_t)nc++;
    out.rows_in = rows;
    out.cols_in = cols;
    out.rank_offset = pivots;
    out.rowptr.assign(1, 0);
    out.colidx.clear();
    out.vals.clear();
    out.row_of.clear();
    out.col_of.assign(nc, 0);
    for (int64_t j = 0; j < cols; j++)
        if (cnew[j] >= 0) out.col_of[cnew[j]] = (int32_t)j;
    for (int64_t i = 0; i < rows; i++) {
        if (rdead[i] || rcnt[i] == 0) continue;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++)
            if (vals[e] != 0 && cnew[colidx[e]] >= 0) {
                out.colidx.push_back(cnew[colidx[e]]);
                out.vals.push_back(vals[e]);
            }
        out.rowptr.push_back((int64_t)out.colidx.size());
        out.row_of.push_back((int32_t)i);
    }
    out.rows = (int64_t)out.row_of.size();
    out.cols = nc;
    return WR_OK;
}

// Locality order (Section 4's "adapted reordering technique"): rows and
// columns renumbered by decreasing entry count, ties by index.  The SpMM
// gathers a block row per entry; in power-law matrices a few columns (and
// the dependent rows) carry most entries, and this packs their block rows
// next to each other, so that the hot ones share cache lines and stay in L1.
wr_status locality_order_host(int64_t rows, int64_t cols, const int64_t *rowptr, const int32_t *colidx,
                              const int32_t *vals, ReducedCsr &out) {
    if (rows < 0 || cols < 0) return fail(WR_EINVAL, "negative size");
    if (!rowptr) return fail(WR_EINVAL, "null row pointer array");
    const int64_t nnz = rowptr[rows];
    if (nnz > 0 && (!colidx || !vals)) return fail(WR_EINVAL, "null column or value array");
    for (int64_t e = 0; e < nnz; e++)
        if (colidx[e] < 0 || colidx[e] >= cols) return fail(WR_EINVAL, "column index out of range");
    std::vector<int64_t> cdeg(cols, 0);
    for (int64_t e = 0; e < nnz; e++) cdeg[colidx[e]]++;
    out.rows_in = out.rows = rows;
    out.cols_in = out.cols = cols;
    out.rank_offset = 0;
    out.row_of.resize(rows);
    out.col_of.resize(cols);
    for (int64_t i = 0; i < rows; i++) out.row_of[i] = (int32_t)i;
    for (int64_t j = 0; j < cols; j++) out.col_of[j] = (int32_t)j;
    std::stable_sort(out.row_of.begin(), out.row_of.end(), [&](int32_t a, int32_t b) {
        return rowptr[a + 1] - rowptr[a] > rowptr[b + 1] - rowptr[b];
    });
    std::stable_sort(out.col_of.begin(), out.col_of.end(), [&](int32_t a, int32_t b) { return cdeg[a] > cdeg[b]; });
    std::vector<int32_t> cnew(cols);
    for (int64_t j = 0; j < cols; j++) cnew[out.col_of[j]] = (int32_t)j;
    out.rowptr.assign(rows + 1, 0);
    out.colidx.resize(nnz);
    out.vals.resize(nnz);
    std::vector<std::pair<int32_t, int32_t>> row;
    int64_t w = 0;
    for (int64_t i = 0; i < rows; i++) {
        const int32_t g = out.row_of[i];
        row.clear();
        for (int64_t e = rowptr[g]; e < rowptr[g + 1]; e++) row.emplace_back(cnew[colidx[e]], vals[e]);
        std::sort(row.begin(), row.end());
        for (const auto &x : row) {
            out.colidx[w] = x.first;
            out.vals[w] = x.second;
            w++;
        }
        out.rowptr[i + 1] = w;
    }
    return WR_OK;
}

}  // namespace wr

using namespace wr;

extern "C" wr_status wr_chain_reduce_csr(int64_t rows, int64_t cols, const int64_t *rowptr, const int32_t *colidx,
                                         const int32_t *vals, int64_t *out_rows, int64_t *out_cols,
                                         int64_t *out_rowptr, int32_t *out_colidx, int32_t *out_vals,
                                         int32_t *out_row_of, int32_t *out_col_of, int64_t *rank_offset) {
    if (!out_rows || !out_cols || !out_rowptr || !rank_offset) return fail(WR_EINVAL, "null output argument");
    ReducedCsr r;
    WR_TRY(chain_reduce_host(rows, cols, rowptr, colidx, vals, r));
    const int64_t nnz = (int64_t)r.colidx.size();
    if (nnz > 0 && (!out_colidx || !out_vals)) return fail(WR_EINVAL, "null output column or value array");
    *out_rows = r.rows;
    *out_cols = r.cols;
    *rank_offset = r.rank_offset;
    std::memcpy(out_rowptr, r.rowptr.data(), sizeof(int64_t) * (r.rows + 1));
    if (nnz > 0) {
        std::memcpy(out_colidx, r.colidx.data(), sizeof(int32_t) * nnz);
        std::memcpy(out_vals, r.vals.data(), sizeof(int32_t) * nnz);
    }
    if (out_row_of && r.rows > 0) std::memcpy(out_row_of, r.row_of.data(), sizeof(int32_t) * r.rows);
    if (out_col_of && r.cols > 0) std::memcpy(out_col_of, r.col_of.data(), sizeof(int32_t) * r.cols);
    return WR_OK;
}

extern "C" wr_status wr_locality_order_csr(int64_t rows, int64_t cols, const int64_t *rowptr, const int32_t *colidx,
                                           const int32_t *vals, int64_t *out_rowptr, int32_t *out_colidx,
                                           int32_t *out_vals, int32_t *out_row_of, int32_t *out_col_of) {
    if (!out_rowptr || !out_row_of || !out_col_of) return fail(WR_EINVAL, "null output argument");
    ReducedCsr r;
    WR_TRY(locality_order_host(rows, cols, rowptr, colidx, vals, r));
    const int64_t nnz = (int64_t)r.colidx.size();
    if (nnz > 0 && (!out_colidx || !out_vals)) return fail(WR_EINVAL, "null output column or value array");
    std::memcpy(out_rowptr, r.rowptr.data(), sizeof(int64_t) * (rows + 1));
    if (nnz > 0) {
        std::memcpy(out_colidx, r.colidx.data(), sizeof(int32_t) * nnz);
        std::memcpy(out_vals, r.vals.data(), sizeof(int32_t) * nnz);
    }
    if (rows > 0) std::memcpy(out_row_of, r.row_of.data(), sizeof(int32_t) * rows);
    if (cols > 0) std::memcpy(out_col_of, r.col_of.data(), sizeof(int32_t) * cols);
    return WR_OK;
}
