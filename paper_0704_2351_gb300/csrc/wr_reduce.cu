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

// Chain reduction along a complex (Section 2.6.4, where a pivot taken in one
// boundary matrix also removes lines of the neighbouring ones).  mats[i] has
// the cells of mats[i+1]'s rows
// as its columns and mats[i] mats[i+1] = 0 over Z.  A unit pivot at (r, c) of
// mats[i] is removed as above (rank offset + 1) and, in the neighbours, the
// line of each shared cell goes too: column r of mats[i-1], row c of
// mats[i+1].  That line is zero or a combination of the others (d o d = 0
// with the pivot's row or column a single +-1), so the neighbours' ranks do
// not change, and the reduced matrices still compose to zero, so the rule
// applies again.  Removals cascade through all the matrices.
namespace {

struct ChainMat {
    int64_t rows = 0, cols = 0;
    const int64_t *rp = nullptr;
    const int32_t *ci = nullptr, *va = nullptr;
    std::vector<int64_t> cptr;
    std::vector<int32_t> crow;
    std::vector<int32_t> rcnt, ccnt;
    std::vector<char> rdead, cdead;
    int64_t pivots = 0;
};

}  // namespace

wr_status chain_reduce_complex_host(int count, wr_csr_io *io) {
    if (count < 1 || !io) return fail(WR_EINVAL, "a complex needs at least one matrix");
    std::vector<ChainMat> M(count);
    for (int i = 0; i < count; i++) {
        ChainMat &a = M[i];
        a.rows = io[i].rows, a.cols = io[i].cols, a.rp = io[i].rowptr, a.ci = io[i].colidx, a.va = io[i].vals;
        if (a.rows < 0 || a.cols < 0 || a.rows >= (int64_t(1) << 31) || a.cols >= (int64_t(1) << 31))
            return fail(WR_EINVAL, "matrix " + std::to_string(i) + ": sizes must be in [0, 2^31)");
        if (!a.rp || a.rp[0] != 0) return fail(WR_EINVAL, "matrix " + std::to_string(i) + ": bad rowptr");
        for (int64_t r = 0; r < a.rows; r++)
            if (a.rp[r + 1] < a.rp[r]) return fail(WR_EINVAL, "matrix " + std::to_string(i) + ": bad rowptr");
        const int64_t nnz = a.rp[a.rows];
        if (nnz > 0 && (!a.ci || !a.va)) return fail(WR_EINVAL, "matrix " + std::to_string(i) + ": null arrays");
        for (int64_t e = 0; e < nnz; e++)
            if (a.ci[e] < 0 || a.ci[e] >= a.cols)
                return fail(WR_EINVAL, "matrix " + std::to_string(i) + ": column index out of range");
        if (i > 0 && M[i - 1].cols != a.rows)
            return fail(WR_EINVAL, "matrix " + std::to_string(i - 1) + "'s columns must be matrix " +
                                       std::to_string(i) + "'s rows");
    }
    // exactness: mats[i] mats[i+1] = 0 over Z (row by row, dense accumulator)
    for (int i = 0; i + 1 < count; i++) {
        const ChainMat &a = M[i], &b = M[i + 1];
        std::vector<__int128> acc(b.cols, 0);  // exact for any int32 entries
        std::vector<int32_t> touched;
        for (int64_t r = 0; r < a.rows; r++) {
            touched.clear();
            for (int64_t e = a.rp[r]; e < a.rp[r + 1]; e++) {
                const int64_t j = a.ci[e], x = a.va[e];
                if (!x) continue;
                for (int64_t f = b.rp[j]; f < b.rp[j + 1]; f++) {
                    if (!b.va[f]) continue;
                    if (acc[b.ci[f]] == 0) touched.push_back(b.ci[f]);
                    acc[b.ci[f]] += (__int128)x * b.va[f];
                }
            }
            bool zero = true;
            for (int32_t c : touched) {
                if (acc[c] != 0) zero = false;
                acc[c] = 0;
            }
            if (!zero)
                return fail(WR_EINVAL, "matrices " + std::to_string(i) + " and " + std::to_string(i + 1) +
                                           " do not compose to zero (not a chain complex)");
        }
    }
    for (ChainMat &a : M) {
        a.rcnt.assign(a.rows, 0);
        a.ccnt.assign(a.cols, 0);
        a.cptr.assign(a.cols + 1, 0);
        for (int64_t r = 0; r < a.rows; r++)
            for (int64_t e = a.rp[r]; e < a.rp[r + 1]; e++)
                if (a.va[e] != 0) {
                    a.rcnt[r]++;
                    a.cptr[a.ci[e] + 1]++;
                }
        for (int64_t j = 0; j < a.cols; j++) {
            a.ccnt[j] = (int32_t)a.cptr[j + 1];
            a.cptr[j + 1] += a.cptr[j];
        }
        a.crow.assign(a.cptr[a.cols], 0);
        std::vector<int64_t> fill(a.cptr.begin(), a.cptr.end() - 1);
        for (int64_t r = 0; r < a.rows; r++)
            for (int64_t e = a.rp[r]; e < a.rp[r + 1]; e++)
                if (a.va[e] != 0) a.crow[fill[a.ci[e]]++] = (int32_t)r;
        a.rdead.assign(a.rows, 0);
        a.cdead.assign(a.cols, 0);
    }
    // work items: (matrix, line, is_row) with a single live entry
    std::deque<std::pair<int, int64_t>> rq, cq;
    for (int i = 0; i < count; i++) {
        for (int64_t r = 0; r < M[i].rows; r++)
            if (M[i].rcnt[r] == 1) rq.emplace_back(i, r);
        for (int64_t j = 0; j < M[i].cols; j++)
            if (M[i].ccnt[j] == 1) cq.emplace_back(i, j);
    }
    auto kill_row = [&](int i, int64_t r) {
        ChainMat &a = M[i];
        if (a.rdead[r]) return;
        a.rdead[r] = 1;
        for (int64_t e = a.rp[r]; e < a.rp[r + 1]; e++) {
            const int64_t c = a.ci[e];
            if (a.va[e] != 0 && !a.cdead[c] && --a.ccnt[c] == 1) cq.emplace_back(i, c);
        }
    };
    auto kill_col = [&](int i, int64_t c) {
        ChainMat &a = M[i];
        if (a.cdead[c]) return;
        a.cdead[c] = 1;
        for (int64_t e = a.cptr[c]; e < a.cptr[c + 1]; e++) {
            const int64_t r = a.crow[e];
            if (!a.rdead[r] && --a.rcnt[r] == 1) rq.emplace_back(i, r);
        }
    };
    auto take = [&](int i, int64_t r, int64_t c) {
        ChainMat &a = M[i];
        a.pivots++;
        a.rdead[r] = 1;  // both lines go before the counts of their crossings drop
        a.cdead[c] = 1;
        for (int64_t e = a.rp[r]; e < a.rp[r + 1]; e++) {
            const int64_t c2 = a.ci[e];
            if (a.va[e] != 0 && !a.cdead[c2] && --a.ccnt[c2] == 1) cq.emplace_back(i, c2);
        }
        for (int64_t e = a.cptr[c]; e < a.cptr[c + 1]; e++) {
            const int64_t r2 = a.crow[e];
            if (!a.rdead[r2] && --a.rcnt[r2] == 1) rq.emplace_back(i, r2);
        }
        if (i > 0) kill_col(i - 1, r);
        if (i + 1 < count) kill_row(i + 1, c);
    };
    while (!rq.empty() || !cq.empty()) {
        while (!rq.empty()) {
            const auto [i, r] = rq.front();
            rq.pop_front();
            ChainMat &a = M[i];
            if (a.rdead[r] || a.rcnt[r] != 1) continue;
            for (int64_t e = a.rp[r]; e < a.rp[r + 1]; e++)
                if (a.va[e] != 0 && !a.cdead[a.ci[e]]) {
                    if (a.va[e] == 1 || a.va[e] == -1) take(i, r, a.ci[e]);
                    break;
                }
        }
        while (!cq.empty()) {
            const auto [i, c] = cq.front();
            cq.pop_front();
            ChainMat &a = M[i];
            if (a.cdead[c] || a.ccnt[c] != 1) continue;
            for (int64_t e = a.cptr[c]; e < a.cptr[c + 1]; e++) {
                const int64_t r = a.crow[e];
                if (a.rdead[r]) continue;
                int32_t v = 0;
                for (int64_t f = a.rp[r]; f < a.rp[r + 1]; f++)
                    if (a.ci[f] == c && a.va[f] != 0) {
                        v = a.va[f];
                        break;
                    }
                if (v == 1 || v == -1) take(i, r, c);
                break;
            }
        }
    }
    // Compact each matrix.  A cell between mats[i] and mats[i+1] (a column of
    // the one, a row of the other) is kept in both while it is live and holds
    // an entry on either side, so that the reduced matrices still compose
    // (out_cols of mats[i] = out_rows of mats[i+1]) and the reduction can run
    // again on its own output; the outer lines (rows of the first matrix,
    // columns of the last) are kept when live and not empty.
    std::vector<std::vector<char>> keep(count > 1 ? count - 1 : 0);
    for (int i = 0; i + 1 < count; i++) {
        const ChainMat &a = M[i], &b = M[i + 1];
        keep[i].assign(a.cols, 0);
        for (int64_t c = 0; c < a.cols; c++)
            keep[i][c] = !a.cdead[c] && !b.rdead[c] && (a.ccnt[c] > 0 || b.rcnt[c] > 0);
    }
    for (int i = 0; i < count; i++) {
        ChainMat &a = M[i];
        wr_csr_io &o = io[i];
        std::vector<int32_t> cnew(a.cols, -1);
        int64_t nc = 0;
        for (int64_t j = 0; j < a.cols; j++)
            if (i + 1 < count ? keep[i][j] != 0 : (!a.cdead[j] && a.ccnt[j] > 0)) {
                if (o.out_col_of) o.out_col_of[nc] = (int32_t)j;
                cnew[j] = (int32_t)nc++;
            }
        int64_t nr = 0, w = 0;
        o.out_rowptr[0] = 0;
        for (int64_t r = 0; r < a.rows; r++) {
            if (i > 0 ? keep[i - 1][r] == 0 : (a.rdead[r] || a.rcnt[r] == 0)) continue;
            for (int64_t e = a.rp[r]; e < a.rp[r + 1]; e++)
                if (a.va[e] != 0 && cnew[a.ci[e]] >= 0) {
                    o.out_colidx[w] = cnew[a.ci[e]];
                    o.out_vals[w] = a.va[e];
                    w++;
                }
            if (o.out_row_of) o.out_row_of[nr] = (int32_t)r;
            o.out_rowptr[++nr] = w;
        }
        o.out_rows = nr;
        o.out_cols = nc;
        o.rank_offset = a.pivots;
    }
    return WR_OK;
}

}  // namespace wr

using namespace wr;

extern "C" wr_status wr_chain_reduce_complex(int32_t count, wr_csr_io *mats) {
    if (!mats) return fail(WR_EINVAL, "null argument");
    for (int i = 0; i < count; i++) {
        const int64_t nnz = mats[i].rowptr ? mats[i].rowptr[std::max<int64_t>(mats[i].rows, 0)] : 0;
        if (!mats[i].out_rowptr || (nnz > 0 && (!mats[i].out_colidx || !mats[i].out_vals)))
            return fail(WR_EINVAL, "matrix " + std::to_string(i) + ": null output arrays");
    }
    return chain_reduce_complex_host(count, mats);
}

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
