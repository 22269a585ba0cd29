/*
 * CPU oracle for the block Wiedemann rank path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct C.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg load this library; the CUDA library
 * never includes, links or calls anything here, and nothing here comes from
 * the CUDA library.
 *
 * Every modular product is formed exactly (unsigned __int128 where needed)
 * and reduced with the C "%" operator.  No blocking, no fusion, no lazy
 * reduction tricks: each function follows the definition or the paper's step
 * order and cites where it comes from (paper: Dumas, Elbaz-Vincent, Giorgi,
 * Urbanska, "Parallel computation of the rank of large sparse matrices from
 * algebraic K-theory", PASCO 2007).
 *
 * Parity pins (what pins each function to something other than itself) are
 * in tests/test_oracle_pins.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

#define OR_GOLDEN 0x9E3779B97F4A7C15ULL

/* allocation count that is never zero */
static size_t nz(int64_t x) { return x > 0 ? (size_t)x : 1; }

/* ------------------------------------------------------------------------ */
/* modular helpers                                                            */
/* ------------------------------------------------------------------------ */

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) {
    return (uint64_t)(((u128)a * (u128)b) % p);
}

static uint64_t addmod(uint64_t a, uint64_t b, uint64_t p) {
    return (uint64_t)(((u128)a + (u128)b) % p);
}

static uint64_t submod(uint64_t a, uint64_t b, uint64_t p) {
    return (uint64_t)(((u128)a + (u128)p - (u128)(b % p)) % p);
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = mulmod(r, a, p);
        a = mulmod(a, a, p);
        e >>= 1;
    }
    return r;
}

/* inverse by Fermat's little theorem (p prime, a != 0 mod p) */
static uint64_t invmod(uint64_t a, uint64_t p) { return powmod(a, p - 2, p); }

/* signed integer -> residue in [0, p) */
static uint64_t residue(int64_t a, uint64_t p) {
    int64_t r = a % (int64_t)p;
    if (r < 0) r += (int64_t)p;
    return (uint64_t)r;
}

uint64_t or_residue(int64_t a, uint64_t p) { return residue(a, p); }
uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t p) { return mulmod(a, b, p); }
uint64_t or_invmod(uint64_t a, uint64_t p) { return invmod(a, p); }

/* ------------------------------------------------------------------------ */
/* primality: deterministic Miller-Rabin for n < 2^32 (bases 2, 7, 61)        */
/* (the paper picks random primes for rank over Q, Section 2.5)               */
/* ------------------------------------------------------------------------ */

int or_is_prime_u32(uint64_t n) {
    if (n < 2) return 0;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (int i = 0; i < 12; i++) {
        if (n == small[i]) return 1;
        if (n % small[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    static const uint64_t bases[] = {2, 7, 61};
    for (int i = 0; i < 3; i++) {
        uint64_t a = bases[i] % n;
        if (a == 0) continue;
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* counter-based random draws (SplitMix64 of Steele, Lea and Flood, 2014)     */
/* The paper draws X, Y and the preconditioner diagonals at random (Section   */
/* 2.5, step 2; Section 2.3); here they are derived from a 64-bit seed:       */
/*   h(seed, tag, idx) = sm(sm(seed ^ tag*GOLDEN) + idx)                      */
/* with sm(x) the SplitMix64 output for state x (x + GOLDEN, then the mix).   */
/* Tags: X = 1, Y = 2, D1 = 3, D2 = 4.  Block entries: h mod p.               */
/* Diagonal entries: 1 + h mod (p - 1), never zero.                            */
/* ------------------------------------------------------------------------ */

uint64_t or_splitmix64(uint64_t x) {
    uint64_t z = x + OR_GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t or_hash(uint64_t seed, uint64_t tag, uint64_t idx) {
    return or_splitmix64(or_splitmix64(seed ^ (tag * OR_GOLDEN)) + idx);
}

/* out[i*width + j] = h(seed, tag, i*width + j) mod p */
void or_derive_block(uint64_t seed, uint64_t tag, int64_t rows, int64_t width, uint64_t p,
                     uint32_t *out) {
    for (int64_t i = 0; i < rows; i++)
        for (int64_t j = 0; j < width; j++) {
            uint64_t idx = (uint64_t)(i * width + j);
            out[idx] = (uint32_t)(or_hash(seed, tag, idx) % p);
        }
}

/* out[i] = 1 + h(seed, tag, i) mod (p - 1) */
void or_derive_diag(uint64_t seed, uint64_t tag, int64_t len, uint64_t p, uint32_t *out) {
    for (int64_t i = 0; i < len; i++)
        out[i] = (uint32_t)(1 + or_hash(seed, tag, (uint64_t)i) % (p - 1));
}

/* ------------------------------------------------------------------------ */
/* sparse products mod p (the black box of Section 1.2: A is only used       */
/* through u -> A u)                                                           */
/* ------------------------------------------------------------------------ */

/* y (rows x w) = A x (cols x w) mod p.  Row-parallel over the host's cores. */
void or_csr_mul(int64_t R, int64_t C, const int64_t *rowptr, const int32_t *colidx,
                const int32_t *vals, uint64_t p, int64_t w, const uint32_t *x, uint32_t *y) {
    (void)C;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < R; i++) {
        for (int64_t b = 0; b < w; b++) {
            u128 acc = 0;
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
                uint64_t a = residue(vals[k], p);
                acc += (u128)a * (u128)x[(int64_t)colidx[k] * w + b];
            }
            y[i * w + b] = (uint32_t)(acc % p);
        }
    }
}

/* Transpose of a CSR matrix by plain counting: (A^T)[j][i] = A[i][j].
 * Outputs rowptr_t (C + 1), colidx_t (nnz), vals_t (nnz). */
void or_csr_transpose(int64_t R, int64_t C, const int64_t *rowptr, const int32_t *colidx,
                      const int32_t *vals, int64_t *rowptr_t, int32_t *colidx_t, int32_t *vals_t) {
    for (int64_t j = 0; j <= C; j++) rowptr_t[j] = 0;
    for (int64_t k = 0; k < rowptr[R]; k++) rowptr_t[colidx[k] + 1]++;
    for (int64_t j = 0; j < C; j++) rowptr_t[j + 1] += rowptr_t[j];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * nz(C));
    for (int64_t j = 0; j < C; j++) fill[j] = rowptr_t[j];
    for (int64_t i = 0; i < R; i++)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
            int64_t j = colidx[k];
            colidx_t[fill[j]] = (int32_t)i;
            vals_t[fill[j]] = vals[k];
            fill[j]++;
        }
    free(fill);
}

typedef struct { int64_t R, C; int64_t *rowptr; int32_t *colidx; int32_t *vals; } csr_t;

static csr_t transpose_alloc(int64_t R, int64_t C, const int64_t *rowptr, const int32_t *colidx,
                             const int32_t *vals) {
    csr_t t;
    int64_t nnz = rowptr[R];
    t.R = C; t.C = R;
    t.rowptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C + 1));
    t.colidx = (int32_t *)malloc(sizeof(int32_t) * nz(nnz));
    t.vals = (int32_t *)malloc(sizeof(int32_t) * nz(nnz));
    or_csr_transpose(R, C, rowptr, colidx, vals, t.rowptr, t.colidx, t.vals);
    return t;
}

static void csr_free(csr_t *t) { free(t->rowptr); free(t->colidx); free(t->vals); }

/* y (cols x w) = A^T x (rows x w) mod p */
void or_csr_tmul(int64_t R, int64_t C, const int64_t *rowptr, const int32_t *colidx,
                 const int32_t *vals, uint64_t p, int64_t w, const uint32_t *x, uint32_t *y) {
    csr_t t = transpose_alloc(R, C, rowptr, colidx, vals);
    or_csr_mul(t.R, t.C, t.rowptr, t.colidx, t.vals, p, w, x, y);
    csr_free(&t);
}

/* diagonal scaling v[i][b] = d[i] * v[i][b] mod p */
static void scale_rows(int64_t n, int64_t w, const uint32_t *d, uint64_t p, uint32_t *v) {
    for (int64_t i = 0; i < n; i++)
        for (int64_t b = 0; b < w; b++)
            v[i * w + b] = (uint32_t)mulmod(d[i], v[i * w + b], p);
}

/*
 * One application of the preconditioned black box (Section 2.3: the
 * preconditioners "are of the form A^T A"; Section 2.5 step 1 "form A~"):
 *   side = 0 (N = C):  v <- D1 A^T D2 A D1 v      (D1: C entries, D2: R entries)
 *   side = 1 (N = R):  v <- D1 A D2 A^T D1 v      (D1: R entries, D2: C entries)
 * v is N x w, row-major.  A is given with its transpose At (or_csr_transpose).
 */
static void blackbox(const csr_t *A, const csr_t *At, uint64_t p, int side, const uint32_t *d1,
                     const uint32_t *d2, int64_t w, uint32_t *v) {
    const csr_t *first = side == 0 ? A : At;   /* maps N-space to the other space */
    const csr_t *second = side == 0 ? At : A;  /* maps it back                    */
    int64_t N = first->C, M = first->R;
    uint32_t *t = (uint32_t *)malloc(sizeof(uint32_t) * nz(N * w));
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * nz(M * w));
    memcpy(t, v, sizeof(uint32_t) * (size_t)(N * w));
    scale_rows(N, w, d1, p, t);                                                     /* D1 v  */
    or_csr_mul(first->R, first->C, first->rowptr, first->colidx, first->vals, p, w, t, u);
    scale_rows(M, w, d2, p, u);                                                     /* D2 .  */
    or_csr_mul(second->R, second->C, second->rowptr, second->colidx, second->vals, p, w, u, v);
    scale_rows(N, w, d1, p, v);                                                     /* D1 .  */
    free(t); free(u);
}

void or_blackbox_apply(int64_t R, int64_t C, const int64_t *rowptr, const int32_t *colidx,
                       const int32_t *vals, uint64_t p, int side, const uint32_t *d1,
                       const uint32_t *d2, int64_t w, uint32_t *v) {
    csr_t A = {R, C, (int64_t *)rowptr, (int32_t *)colidx, (int32_t *)vals};
    csr_t At = transpose_alloc(R, C, rowptr, colidx, vals);
    blackbox(&A, &At, p, side, d1, d2, w, v);
    csr_free(&At);
}

/* S (m x n) = X^T V mod p; X: N x m, V: N x n */
void or_project(int64_t N, int64_t m, int64_t n, const uint32_t *X, const uint32_t *V, uint64_t p,
                uint32_t *S) {
    for (int64_t a = 0; a < m; a++)
        for (int64_t b = 0; b < n; b++) {
            u128 acc = 0;
            for (int64_t i = 0; i < N; i++) acc += (u128)X[i * m + a] * (u128)V[i * n + b];
            S[a * n + b] = (uint32_t)(acc % p);
        }
}

/*
 * Block Wiedemann sequence (Section 2.2 and Section 2.5 step 2):
 *   S_i = X^T A~^i Y mod p, i = 0 .. L-1, S laid out [i][a][b] (L x m x n).
 * Literal definition: v <- Y; for each i: S_i = X^T v; v <- A~ v.
 * If V_out is non-null, the final v (= A~^(L-1) Y) is written there.
 */
void or_sequence(int64_t R, int64_t C, const int64_t *rowptr, const int32_t *colidx,
                 const int32_t *vals, uint64_t p, int side, const uint32_t *d1, const uint32_t *d2,
                 int64_t m, int64_t n, const uint32_t *X, const uint32_t *Y, int64_t L, uint32_t *S,
                 uint32_t *V_out) {
    int64_t N = side == 0 ? C : R;
    csr_t A = {R, C, (int64_t *)rowptr, (int32_t *)colidx, (int32_t *)vals};
    csr_t At = transpose_alloc(R, C, rowptr, colidx, vals);
    uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * nz(N * n));
    memcpy(v, Y, sizeof(uint32_t) * (size_t)(N * n));
    for (int64_t i = 0; i < L; i++) {
        or_project(N, m, n, X, v, p, S + i * m * n);
        if (i + 1 < L) blackbox(&A, &At, p, side, d1, d2, n, v);
    }
    if (V_out) memcpy(V_out, v, sizeof(uint32_t) * (size_t)(N * n));
    free(v);
    csr_free(&At);
}

/* ------------------------------------------------------------------------ */
/* rank by Gaussian elimination mod p: the plain definition of rank_p(A)      */
/* (the paper uses elimination mod p for the smaller matrices, Section 2.6.3) */
/* ------------------------------------------------------------------------ */

/* dense: a is rows x cols row-major (any int64 values); destroyed. */
int64_t or_rank_dense(int64_t rows, int64_t cols, int64_t *a, uint64_t p) {
    for (int64_t k = 0; k < rows * cols; k++) a[k] = (int64_t)residue(a[k], p);
    int64_t rank = 0;
    for (int64_t c = 0; c < cols && rank < rows; c++) {
        int64_t piv = -1;
        for (int64_t i = rank; i < rows; i++)
            if (a[i * cols + c] != 0) { piv = i; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int64_t j = 0; j < cols; j++) {
                int64_t tmp = a[piv * cols + j];
                a[piv * cols + j] = a[rank * cols + j];
                a[rank * cols + j] = tmp;
            }
        uint64_t inv = invmod((uint64_t)a[rank * cols + c], p);
        for (int64_t i = rank + 1; i < rows; i++) {
            uint64_t f = mulmod((uint64_t)a[i * cols + c], inv, p);
            if (f == 0) continue;
            for (int64_t j = c; j < cols; j++)
                a[i * cols + j] = (int64_t)submod((uint64_t)a[i * cols + j],
                                                  mulmod(f, (uint64_t)a[rank * cols + j], p), p);
        }
        rank++;
    }
    return rank;
}

/* determinant of a dense n x n matrix of residues mod p (destroyed) */
uint64_t or_det_dense(int64_t n, uint64_t *a, uint64_t p) {
    uint64_t det = 1 % p;
    for (int64_t c = 0; c < n; c++) {
        int64_t piv = -1;
        for (int64_t i = c; i < n; i++)
            if (a[i * n + c] % p != 0) { piv = i; break; }
        if (piv < 0) return 0;
        if (piv != c) {
            for (int64_t j = 0; j < n; j++) {
                uint64_t tmp = a[piv * n + j]; a[piv * n + j] = a[c * n + j]; a[c * n + j] = tmp;
            }
            det = submod(0, det, p);
        }
        det = mulmod(det, a[c * n + c], p);
        uint64_t inv = invmod(a[c * n + c], p);
        for (int64_t i = c + 1; i < n; i++) {
            uint64_t f = mulmod(a[i * n + c], inv, p);
            if (f == 0) continue;
            for (int64_t j = c; j < n; j++)
                a[i * n + j] = submod(a[i * n + j], mulmod(f, a[c * n + j], p), p);
        }
    }
    return det;
}

/* sparse rows as growable (col, val) arrays sorted by col */
typedef struct { int64_t len, cap; int32_t *col; uint32_t *val; } srow;

static void srow_free(srow *r) { free(r->col); free(r->val); r->col = NULL; r->val = NULL; r->len = r->cap = 0; }

/* out = r - f * q  (mod p), sparse merge */
static void srow_axpy(srow *out, const srow *r, uint64_t f, const srow *q, uint64_t p) {
    int64_t cap = r->len + q->len;
    out->col = (int32_t *)malloc(sizeof(int32_t) * nz(cap));
    out->val = (uint32_t *)malloc(sizeof(uint32_t) * nz(cap));
    out->cap = cap;
    int64_t i = 0, j = 0, k = 0;
    while (i < r->len || j < q->len) {
        int32_t c;
        uint64_t v;
        if (j >= q->len || (i < r->len && r->col[i] < q->col[j])) {
            c = r->col[i]; v = r->val[i]; i++;
        } else if (i >= r->len || q->col[j] < r->col[i]) {
            c = q->col[j]; v = submod(0, mulmod(f, q->val[j], p), p); j++;
        } else {
            c = r->col[i]; v = submod(r->val[i], mulmod(f, q->val[j], p), p); i++; j++;
        }
        if (v != 0) { out->col[k] = c; out->val[k] = (uint32_t)v; k++; }
    }
    out->len = k;
}

/*
 * Sparse elimination mod p: rows are taken in order of increasing nonzero
 * count (fewest first, a Markowitz-style choice) and inserted into a row
 * echelon basis: a row is reduced by the basis row owning its leading column
 * until its leading column is free; it then joins the basis.  The rank is the
 * number of basis rows.
 */
int64_t or_rank_sparse(int64_t R, int64_t C, const int64_t *rowptr, const int32_t *colidx,
                       const int32_t *vals, uint64_t p) {
    srow *piv = (srow *)calloc((size_t)C + 1, sizeof(srow));
    char *has = (char *)calloc((size_t)C + 1, 1);
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * nz(R));
    for (int64_t i = 0; i < R; i++) order[i] = i;
    /* order rows by nnz (insertion sort would be O(R^2); counting sort) */
    int64_t maxlen = 0;
    for (int64_t i = 0; i < R; i++) {
        int64_t l = rowptr[i + 1] - rowptr[i];
        if (l > maxlen) maxlen = l;
    }
    int64_t *cnt = (int64_t *)calloc((size_t)maxlen + 2, sizeof(int64_t));
    for (int64_t i = 0; i < R; i++) cnt[rowptr[i + 1] - rowptr[i] + 1]++;
    for (int64_t l = 0; l <= maxlen; l++) cnt[l + 1] += cnt[l];
    for (int64_t i = 0; i < R; i++) order[cnt[rowptr[i + 1] - rowptr[i]]++] = i;
    free(cnt);

    int64_t rank = 0;
    for (int64_t t = 0; t < R; t++) {
        int64_t i = order[t];
        /* load row i as residues, sorted by column, duplicates summed */
        int64_t l = rowptr[i + 1] - rowptr[i];
        srow cur;
        cur.len = 0; cur.cap = l;
        cur.col = (int32_t *)malloc(sizeof(int32_t) * nz(l));
        cur.val = (uint32_t *)malloc(sizeof(uint32_t) * nz(l));
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
            /* insertion into sorted position */
            int32_t c = colidx[k];
            uint64_t v = residue(vals[k], p);
            int64_t pos = cur.len;
            while (pos > 0 && cur.col[pos - 1] > c) pos--;
            if (pos > 0 && cur.col[pos - 1] == c) {
                cur.val[pos - 1] = (uint32_t)addmod(cur.val[pos - 1], v, p);
            } else {
                memmove(cur.col + pos + 1, cur.col + pos, sizeof(int32_t) * (size_t)(cur.len - pos));
                memmove(cur.val + pos + 1, cur.val + pos, sizeof(uint32_t) * (size_t)(cur.len - pos));
                cur.col[pos] = c; cur.val[pos] = (uint32_t)v; cur.len++;
            }
        }
        /* drop zeros */
        int64_t k2 = 0;
        for (int64_t k = 0; k < cur.len; k++)
            if (cur.val[k]) { cur.col[k2] = cur.col[k]; cur.val[k2] = cur.val[k]; k2++; }
        cur.len = k2;
        /* reduce by basis rows on the leading column */
        while (cur.len > 0 && has[cur.col[0]]) {
            int32_t c = cur.col[0];
            uint64_t f = cur.val[0];  /* basis row is normalised: leading value 1 */
            srow nxt;
            srow_axpy(&nxt, &cur, f, &piv[c], p);
            srow_free(&cur);
            cur = nxt;
        }
        if (cur.len > 0) {
            uint64_t inv = invmod(cur.val[0], p);
            for (int64_t k = 0; k < cur.len; k++) cur.val[k] = (uint32_t)mulmod(cur.val[k], inv, p);
            piv[cur.col[0]] = cur;
            has[cur.col[0]] = 1;
            rank++;
        } else {
            srow_free(&cur);
        }
    }
    for (int64_t c = 0; c <= C; c++) if (has[c]) srow_free(&piv[c]);
    free(piv); free(has); free(order);
    return rank;
}

/* ------------------------------------------------------------------------ */
/* scalar generator: Berlekamp-Massey (Wiedemann's algorithm, Section 1.2)    */
/* Returns the linear complexity Lc and the connection polynomial             */
/* conn[0..Lc] (conn[0] = 1) with s_i + sum_{j=1..Lc} conn[j] s_{i-j} = 0 for */
/* Lc <= i < len.  conn must hold len+1 entries.                               */
/* ------------------------------------------------------------------------ */

int64_t or_berlekamp_massey(const uint32_t *s, int64_t len, uint64_t p, uint32_t *conn) {
    uint64_t *Cp = (uint64_t *)calloc((size_t)len + 1, sizeof(uint64_t));
    uint64_t *Bp = (uint64_t *)calloc((size_t)len + 1, sizeof(uint64_t));
    uint64_t *Tp = (uint64_t *)calloc((size_t)len + 1, sizeof(uint64_t));
    Cp[0] = 1; Bp[0] = 1;
    int64_t Lc = 0, shift = 1;
    uint64_t b = 1;
    for (int64_t i = 0; i < len; i++) {
        uint64_t d = s[i] % p;
        for (int64_t j = 1; j <= Lc; j++) d = addmod(d, mulmod(Cp[j], s[i - j], p), p);
        if (d == 0) { shift++; continue; }
        uint64_t coef = mulmod(d, invmod(b, p), p);
        if (2 * Lc <= i) {
            memcpy(Tp, Cp, sizeof(uint64_t) * (size_t)(len + 1));
            for (int64_t j = 0; j + shift <= len; j++)
                Cp[j + shift] = submod(Cp[j + shift], mulmod(coef, Bp[j], p), p);
            Lc = i + 1 - Lc;
            memcpy(Bp, Tp, sizeof(uint64_t) * (size_t)(len + 1));
            b = d;
            shift = 1;
        } else {
            for (int64_t j = 0; j + shift <= len; j++)
                Cp[j + shift] = submod(Cp[j + shift], mulmod(coef, Bp[j], p), p);
            shift++;
        }
    }
    for (int64_t j = 0; j <= len; j++) conn[j] = (uint32_t)Cp[j];
    free(Cp); free(Bp); free(Tp);
    return Lc;
}

/* ------------------------------------------------------------------------ */
/* sigma-basis by M-Basis (Giorgi, Jeannerod, Villard, ISSAC 2003; the paper  */
/* computes the minimal matrix generator through sigma-bases, Section 2.4,    */
/* "sigma-basis computations", and Section 2.5 step 3).                        */
/*                                                                             */
/* Input: S_0..S_{L-1} (m x n).  H(x) = [ S(x) | -I_m ] (m x q, q = m + n).    */
/* Output: M(x) (q x q, coefficients M[t][r][c], t <= Dcap) with               */
/*   H(x) M(x) = 0 mod x^L, minimal for the shift s = (0^n, 1^m),              */
/* and the shifted column degrees deg[c].                                      */
/*                                                                             */
/* Order k (k = 0 .. L-1):                                                     */
/*   1. discrepancy  Delta = coeff of x^k in H M (m x q)                       */
/*   2. columns sorted by (deg, index) ascending                               */
/*   3. in that order, each column is reduced by the pivots found so far:      */
/*      for each pivot (c, r) in order of creation, if Delta[r][j] != 0:       */
/*      col_j -= (Delta[r][j] / Delta[r][c]) col_c  (on Delta and on M);       */
/*      if Delta_j is still nonzero, j becomes a pivot with pivot row          */
/*      r = the first row where Delta_j is nonzero                              */
/*   4. every pivot column is multiplied by x: deg += 1                        */
/* ------------------------------------------------------------------------ */

int or_mbasis(const uint32_t *S, int64_t L, int64_t m, int64_t n, uint64_t p, int64_t Dcap,
              uint32_t *M, int32_t *deg) {
    int64_t q = m + n;
    int64_t QQ = q * q;
    memset(M, 0, sizeof(uint32_t) * (size_t)((Dcap + 1) * QQ));
    for (int64_t c = 0; c < q; c++) {
        M[c * q + c] = 1;
        deg[c] = c < n ? 0 : 1;
    }
    uint64_t *delta = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m * q));
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)q);
    int64_t *pcol = (int64_t *)malloc(sizeof(int64_t) * (size_t)q);
    int64_t *prow = (int64_t *)malloc(sizeof(int64_t) * (size_t)q);
    for (int64_t k = 0; k < L; k++) {
        /* 1. discrepancy */
        for (int64_t c = 0; c < q; c++) {
            for (int64_t a = 0; a < m; a++) {
                u128 acc = 0;
                int64_t tmax = deg[c] < k ? deg[c] : k;
                for (int64_t t = 0; t <= tmax; t++)
                    for (int64_t r = 0; r < n; r++)
                        acc += (u128)S[((k - t) * m + a) * n + r] * (u128)M[(t * q + r) * q + c];
                uint64_t v = (uint64_t)(acc % p);
                if (k <= Dcap) v = submod(v, M[(k * q + (n + a)) * q + c], p);
                delta[a * q + c] = v;
            }
        }
        /* 2. order by (deg, index): stable insertion sort */
        for (int64_t c = 0; c < q; c++) ord[c] = c;
        for (int64_t i = 1; i < q; i++) {
            int64_t c = ord[i], j = i;
            while (j > 0 && deg[ord[j - 1]] > deg[c]) { ord[j] = ord[j - 1]; j--; }
            ord[j] = c;
        }
        /* 3. elimination */
        int64_t np = 0;
        for (int64_t oi = 0; oi < q; oi++) {
            int64_t j = ord[oi];
            for (int64_t t = 0; t < np; t++) {
                int64_t c = pcol[t], r = prow[t];
                if (delta[r * q + j] == 0) continue;
                uint64_t lam = mulmod(delta[r * q + j], invmod(delta[r * q + c], p), p);
                for (int64_t a = 0; a < m; a++)
                    delta[a * q + j] = submod(delta[a * q + j], mulmod(lam, delta[a * q + c], p), p);
                for (int64_t tt = 0; tt <= deg[c] && tt <= Dcap; tt++)
                    for (int64_t rr = 0; rr < q; rr++) {
                        uint32_t *dst = &M[(tt * q + rr) * q + j];
                        *dst = (uint32_t)submod(*dst, mulmod(lam, M[(tt * q + rr) * q + c], p), p);
                    }
            }
            int64_t r0 = -1;
            for (int64_t a = 0; a < m; a++)
                if (delta[a * q + j] != 0) { r0 = a; break; }
            if (r0 >= 0) { pcol[np] = j; prow[np] = r0; np++; }
        }
        /* 4. multiply pivot columns by x */
        for (int64_t t = 0; t < np; t++) {
            int64_t c = pcol[t];
            if (deg[c] + 1 > Dcap) { free(delta); free(ord); free(pcol); free(prow); return -1; }
            for (int64_t tt = deg[c]; tt >= 0; tt--)
                for (int64_t rr = 0; rr < q; rr++)
                    M[((tt + 1) * q + rr) * q + c] = M[(tt * q + rr) * q + c];
            for (int64_t rr = 0; rr < q; rr++) M[rr * q + c] = 0;
            deg[c] += 1;
        }
    }
    free(delta); free(ord); free(pcol); free(prow);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* x-adic valuation of det G for a polynomial matrix G (n x n, coefficients   */
/* G[t][i][j], t < T), by Gaussian elimination over F_p[[x]] / x^T: the pivot  */
/* is an entry of least valuation v; it is a unit times x^v, every other row  */
/* is reduced by a power-series multiple of the pivot row, and the precision  */
/* drops by v.  Returns the valuation, or -1 when the precision runs out.      */
/* (The paper needs codeg det F, Section 2.5 step 4.)                          */
/* ------------------------------------------------------------------------ */

int64_t or_det_valuation(const uint32_t *G, int64_t n, int64_t T, uint64_t p) {
    uint64_t *g = (uint64_t *)malloc(sizeof(uint64_t) * nz(n * n * T));
    /* g[(i*n + j)*T + t] */
    for (int64_t t = 0; t < T; t++)
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++) g[(i * n + j) * T + t] = G[(t * n + i) * n + j] % p;
    char *rdone = (char *)calloc((size_t)n + 1, 1);
    char *cdone = (char *)calloc((size_t)n + 1, 1);
    uint64_t *ser = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(T + 1));
    uint64_t *inv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(T + 1));
    uint64_t *mu = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(T + 1));
    int64_t prec = T, total = 0;
    for (int64_t step = 0; step < n; step++) {
        int64_t bi = -1, bj = -1, bv = prec;
        for (int64_t i = 0; i < n; i++) {
            if (rdone[i]) continue;
            for (int64_t j = 0; j < n; j++) {
                if (cdone[j]) continue;
                for (int64_t t = 0; t < bv; t++)
                    if (g[(i * n + j) * T + t]) { bv = t; bi = i; bj = j; break; }
            }
        }
        if (bi < 0) { total = -1; break; }
        total += bv;
        int64_t np_ = prec - bv;           /* new precision */
        /* unit part of the pivot: u = pivot / x^bv, inverse mod x^np_ */
        for (int64_t t = 0; t < np_; t++) ser[t] = g[(bi * n + bj) * T + bv + t];
        inv[0] = invmod(ser[0], p);
        for (int64_t t = 1; t < np_; t++) {
            u128 acc = 0;
            for (int64_t s = 1; s <= t; s++) acc += (u128)ser[s] * inv[t - s];
            inv[t] = mulmod(submod(0, (uint64_t)(acc % p), p), inv[0], p);
        }
        for (int64_t i = 0; i < n; i++) {
            if (rdone[i] || i == bi) continue;
            /* mu = (g[i][bj] / x^bv) * inv  mod x^np_ */
            for (int64_t t = 0; t < np_; t++) {
                u128 acc = 0;
                for (int64_t s = 0; s <= t; s++) acc += (u128)g[(i * n + bj) * T + bv + s] * inv[t - s];
                mu[t] = (uint64_t)(acc % p);
            }
            for (int64_t j = 0; j < n; j++) {
                if (cdone[j]) continue;
                for (int64_t t = np_ - 1; t >= 0; t--) {
                    u128 acc = 0;
                    for (int64_t s = 0; s <= t; s++) acc += (u128)mu[s] * g[(bi * n + j) * T + t - s];
                    g[(i * n + j) * T + t] = submod(g[(i * n + j) * T + t], (uint64_t)(acc % p), p);
                }
                for (int64_t t = np_; t < T; t++) g[(i * n + j) * T + t] = 0;
            }
        }
        rdone[bi] = 1; cdone[bj] = 1;
        prec = np_;
    }
    free(g); free(rdone); free(cdone); free(ser); free(inv); free(mu);
    return total;
}

/* det of a polynomial matrix evaluated at x0: G[t][i][j], t <= D */
uint64_t or_det_poly_eval(const uint32_t *G, int64_t n, int64_t D, uint64_t x0, uint64_t p) {
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * nz(n * n));
    for (int64_t i = 0; i < n * n; i++) {
        uint64_t acc = 0;
        for (int64_t t = D; t >= 0; t--) acc = addmod(mulmod(acc, x0, p), G[t * n * n + i], p);
        a[i] = acc;
    }
    uint64_t d = or_det_dense(n, a, p);
    free(a);
    return d;
}
