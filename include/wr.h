/*
 * wr.h -- exact rank of large sparse integer matrices modulo a prime p, by
 * block Wiedemann, on one GB300 GPU (sm_103a).
 *
 * Method (Dumas, Elbaz-Vincent, Giorgi, Urbanska, "Parallel computation of the
 * rank of large sparse matrices from algebraic K-theory", PASCO 2007):
 * Section 2.5, "Block Wiedemann Rank Algorithm":
 *   1. form A~ from A with preconditioners of the form A^T A (Section 2.3):
 *      A~ = D1 A^T D2 A D1 (N = cols) or D1 A D2 A^T D1 (N = rows), D1, D2
 *      random nonsingular diagonals;
 *   2. the sequence S_i = X^T A~^i Y, i = 0 .. L-1 (Section 2.2, Coppersmith's
 *      block Wiedemann), L = ceil(N/m) + ceil(N/n) + 2 by default;
 *   3. the minimal matrix generator F of {S_i} through a sigma-basis
 *      (Section 2.4, "sigma-basis computations"; M-Basis of Giorgi, Jeannerod,
 *      Villard);
 *   4. r = deg det F - codeg det F.
 * Rank over Q: the maximum of the ranks modulo several primes (Section 2.5,
 * last paragraph).
 *
 * Conventions for every call:
 *   - every function returns wr_status (WR_OK = 0, errors < 0) or a plain
 *     value documented with it; no call aborts or traps; wr_last_error()
 *     gives a message for the last failing call of the calling thread;
 *   - host pointers are read (or written) during the call only and stay
 *     owned by the caller; device pointers (names starting with d_) must be
 *     memory of the context's device, also owned by the caller;
 *   - matrices, results and servers are opaque and owned by the library
 *     until the matching *_free / *_stop call;
 *   - residues are uint32 in [0, p); blocks are row-major; the sequence is
 *     laid out [i][a][b] (L x m x n); generator coefficients [k][row][col];
 *   - all work is queued on the context's stream; calls that return host
 *     values synchronise that stream.
 */
#ifndef WR_H
#define WR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WR_OK = 0,
    WR_EINVAL = -1,      /* bad argument (null pointer, size, block width ...)      */
    WR_ENOMEM = -2,      /* device or host allocation failed                        */
    WR_EDEVICE = -3,     /* CUDA error; message from the runtime                    */
    WR_ETIMEDOUT = -4,   /* a bounded device or host wait ran out                   */
    WR_ENOTPRIME = -5,   /* p is not a prime with 2 < p < 2^31                       */
    WR_EOVERFLOW = -6,   /* an entry or a size does not fit the exact formats       */
    WR_EPROBFAIL = -7,   /* Monte Carlo failure detected (singular generator ...);   */
                         /* retry with another seed                                 */
    WR_EBUSY = -8        /* server queue full / resource busy                       */
} wr_status;

enum { WR_PROJ_GENERIC = 0, WR_PROJ_SYMMETRIC = 1 };
enum { WR_SIDE_AUTO = -1, WR_SIDE_COLS = 0, WR_SIDE_ROWS = 1 };
enum { WR_WANT_SEQUENCE = 1, WR_WANT_GENERATOR = 2 };

typedef struct wr_ctx wr_ctx;
typedef struct wr_matrix wr_matrix;
typedef struct wr_result wr_result;
typedef struct wr_server wr_server;

/* Parameters of one rank computation; copied on call. */
typedef struct {
    uint32_t prime;      /* 2 < p < 2^31, checked by deterministic Miller-Rabin           */
    uint32_t m, n;       /* block sizes, 1..32 each; m = n = 1 is scalar Wiedemann        */
    uint64_t seed;       /* derives X, Y, D1, D2: h(seed, tag, idx) = sm(sm(seed ^ tag*G) */
                         /* + idx) with sm = SplitMix64 output, G = 0x9E3779B97F4A7C15;   */
                         /* X, Y entries h mod p (tags 1, 2; idx = row*width + col);      */
                         /* D1, D2 entries 1 + h mod (p - 1) (tags 3, 4; idx = row)       */
    int32_t projection;  /* WR_PROJ_GENERIC (X independent) or WR_PROJ_SYMMETRIC (X = Y,  */
                         /* m = n; Section 2.3)                                           */
    int32_t side;        /* WR_SIDE_AUTO (N = min(rows, cols)), WR_SIDE_COLS, WR_SIDE_ROWS */
    uint64_t seq_len;    /* 0: L = ceil(N/m) + ceil(N/n) + 2                               */
    uint32_t want;       /* WR_WANT_SEQUENCE | WR_WANT_GENERATOR: keep them in the result */
} wr_params;

/* Phase times of the last wr_rank on a context (milliseconds, CUDA events). */
typedef struct {
    double setup_ms;     /* X, Y, D1, D2 derivation and preconditioning set-up             */
    double sequence_ms;  /* the black-box applications and projections (two terms each for */
                         /* the symmetric projection and the generic one with m = n)     */
    double sigma_ms;     /* sigma-basis, from its start to its end (host clock)           */
    double readout_ms;   /* generator selection, det valuations, rank                     */
    double total_ms;
    double spmm_ms;      /* when profiling is on: summed duration of the sampled SpMM      */
    int64_t spmm_launches; /* launches those samples cover                                  */
    double spmm_bytes;   /* algorithmic bytes of those launches                            */
    int64_t kernel_launches; /* kernels launched through this context since its creation  */
                             /* (each replay of a captured graph counts its kernel nodes)    */
    double sigma_window_ms;  /* when profiling is on: sigma-basis time in the discrepancy    */
    double sigma_local_ms;   /* windows, the per-chunk M-Basis and the transform products    */
    double sigma_apply_ms;
    double sigma_tail_ms;    /* sigma-basis time after the sequence's end: with the pipeline  */
                             /* (wr_set_pipeline) sigma_ms overlaps the sequence and only    */
                             /* this part adds to the time to rank                           */
    int64_t sequence_terms;  /* terms the sequence computed (early termination: at least the */
                             /* result's seq_len, the terms the generator used)               */
    double sigma_product_ms; /* when profiling is on: PM-Basis polynomial matrix products   */
                             /* (residuals and basis products, CUDA events)                  */
} wr_timings;

/* Device allocator callbacks (for example PyTorch's caching allocator):
 * alloc(bytes, stream, user) returns device memory usable on `stream` (the
 * context's stream) or NULL; release(ptr, bytes, stream, user) gives it back,
 * in stream order (work already queued on `stream` may still use it). */
typedef void *(*wr_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*wr_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to
 * queue work on (for example a torch stream), or NULL for a stream owned by
 * the context.  (The paper's Section 3.1 runs one process per column of Y; on
 * one GPU every column of the block goes through one kernel pass instead.) */
wr_status wr_create(wr_ctx **out, int device, void *cuda_stream);
void wr_destroy(wr_ctx *ctx);
/* Message of the last failing call made by this thread ("" if none). */
const char *wr_last_error(void);
/* Turn per-kernel CUDA-event sampling of the SpMM passes on (1) or off (0). */
wr_status wr_set_profiling(wr_ctx *ctx, int on);
wr_status wr_last_timings(const wr_ctx *ctx, wr_timings *out);
/* Orders per chunk of the blocked sigma-basis (1..64; 0 = automatic).  The
 * result does not depend on it; the time does: each chunk runs its M-Basis
 * steps in one thread block, whose work per order grows with the chunk, while
 * the discrepancy and product kernels around it do the same total work for
 * any chunk size and cost a few launches per chunk. */
wr_status wr_set_sigma_chunk(wr_ctx *ctx, int32_t orders);
/* Sigma-bases of more than `orders` orders (>= 64) are computed by PM-Basis
 * (Section 2.4): halved recursively down to leaves of at most `orders`
 * orders, which run the blocked M-Basis, with the residuals and the products
 * of the halves' bases done as polynomial matrix products by number-theoretic
 * transforms over three FFT primes and the CRT.  The result is the same basis
 * bit for bit; a leaf as large as the sequence turns PM-Basis off.  0
 * (default) = automatic: PM-Basis with 8,192-order leaves for sequences longer
 * than 131,072 orders when m + n <= 32, with 512-order leaves for sequences
 * longer than 2,048 orders when m + n > 32, the blocked M-Basis otherwise.
 * With the pipeline (wr_set_pipeline) PM-Basis trails the sequence in
 * segments, each about half of the orders still to come but at most a
 * quarter of all (down to two leaves): a segment's residual against the
 * basis so far, its own basis and
 * the product start as soon as its terms are published, so that one short
 * segment is left when the sequence ends; the M-Basis trails it chunk by
 * chunk. */
wr_status wr_set_sigma_leaf(wr_ctx *ctx, int64_t orders);
/* SpMM tile shape: the residues each lane gathers from a row of the dense
 * block (1, 2, 4 or 8; the row's n residues are spread over n / that many
 * lanes, at most 32), plus 16 for the streaming cache hints (the matrix's
 * entries and the output rows are loaded and stored evict-first, so that L2
 * keeps rows of the gathered block).
 * With autotuning on (default), the first sequence or black-box application
 * on a matrix with at least 2^20 stored entries times each candidate (every
 * lane width, with and without the hints) on that matrix's two layouts (a few
 * launches each, CUDA events) and keeps the
 * fastest, per matrix, layout and block width; smaller matrices and autotune
 * off use the default (2 residues for n <= 8, 4 above).  wr_set_lane_width
 * forces one (0 = tuned or default).  Results never depend on it. */
wr_status wr_set_autotune(wr_ctx *ctx, int32_t on);
/* Route the context's device allocations through the caller's allocator
 * (both callbacks, or NULL, NULL for the default stream-ordered pool).
 * Matrices keep the allocator they were loaded with until wr_matrix_free;
 * batch and server slots inherit the context's callbacks, which may then be
 * called from the library's worker threads. */
wr_status wr_set_allocator(wr_ctx *ctx, wr_alloc_fn alloc, wr_free_fn release, void *user);
wr_status wr_set_lane_width(wr_ctx *ctx, int32_t residues);
/* wr_rank pipeline (on by default): the sigma-basis trails the sequence on a
 * second stream driven by a second host thread.  M-Basis orders k .. k+b-1
 * need only S_0 .. S_{k+b-1} (Section 2.4's sigma-basis is computed order by
 * order), so each chunk starts as soon as the sequence has produced its terms
 * and the two phases overlap on the device.  Results do not depend on it.
 * mode 0: off (the sigma-basis after the sequence); 2: on, the
 * sigma-basis's stream at the greatest priority (it keeps up with the terms
 * as they are published and the SpMM takes the rest of the device); 3: on,
 * the sequence's stream at the greatest priority (its SpMM blocks go first,
 * the sigma-basis fills the gaps); 1 (default): on, 2 when the sigma-basis
 * trails in PM-Basis segments (whose kernels need most of an SM and would
 * fall behind) and 3 when the blocked M-Basis trails chunk by chunk.  Other
 * values: WR_EINVAL. */
wr_status wr_set_pipeline(wr_ctx *ctx, int32_t mode);
/* Early termination of wr_rank (off by default; orders = 0).  The trailing
 * M-Basis watches the generator candidates (the n basis columns of smallest
 * shifted degree); once they have had zero discrepancy for `orders`
 * consecutive orders (counted per whole chunk) the generator is taken as
 * stable, the sequence stops and the rank is read from the basis so far,
 * instead of after L = ceil(N/m) + ceil(N/n) + 2 terms (about 2r/n + O(1)
 * terms suffice for rank r: the iteration count 2 + 2r/p of Table
 * tab:r-time; Section 4 remarks that early termination needs the
 * order-by-order basis, which is what runs here).  A false
 * stop needs orders * m random residues to vanish; 64 is a sensible value.
 * Needs the pipeline (wr_set_pipeline); the result's seq_len and sequence
 * then hold the terms actually used, and the run always uses M-Basis. */
wr_status wr_set_early_termination(wr_ctx *ctx, int64_t orders);
/* Generic projection with m = n (on by default): A~ = D1 A^T D2 A D1 is
 * symmetric, so with U_k = A~^k X and V_k = A~^k Y the terms are
 * S_2k = U_k^T V_k and S_2k+1 = (A D1 U_k)^T D2 (A D1 V_k) (A~ symmetric:
 * Section 2.3).  X and Y are then carried side by side in one block of width 2n
 * (n <= 32: rows of up to 64 residues) and one black-box application yields
 * two terms.  Off: one term per
 * application on a block of width n.  The sequence is the same either way. */
wr_status wr_set_paired_projection(wr_ctx *ctx, int32_t on);
/* Gram projections beside the passes (off by default): with two terms per
 * application (the symmetric projection, or the paired generic one) the
 * Gram product of W = D2 A D1 V_k runs on a second stream beside the pass
 * that produces the next T, and the Gram product of T beside the next
 * application's first pass; each pass waits only for the Gram product that
 * still reads the buffer it overwrites, and every group of applications
 * joins the sequence stream at its end.  The sequence is the same either
 * way (Section 2.3's terms, summed in the same order).  Measured on GB300 on
 * the 1.9M x 1.95M block-32 matrix it is slower: the Gram products take SM
 * resources from the SpMM's gathers and stream their rows through the L2 that
 * holds the gathered block (a width-32 pass 741 -> 940 us; with the Gram
 * grid capped at half a block per SM 1,257 us), which costs more than the
 * Gram products it hides. */
wr_status wr_set_projection_overlap(wr_ctx *ctx, int32_t on);
/* Where the Gram projections run (the terms of the symmetric projection and of
 * the paired generic one, Section 2.3; Table tab:r-opp col. 3 is the paper's
 * dot-product step): 1 = the tensor cores, 0 = 64-bit integer multiply-adds,
 * -1 (default) = the tensor cores for blocks of 16 columns and more (m, n >=
 * 16), the integer path below.  The tensor-core path is exact: every residue
 * is split into four balanced 8-bit digits (bf16 values), tcgen05 MMAs sum the
 * 16 digit products per residue product in fp32 over at most 512 rows (every
 * partial sum an integer below 2^23), and the sums are drained into int64 and
 * recombined mod p.  The result is the same bit for bit either way. */
wr_status wr_set_tensor_projection(wr_ctx *ctx, int32_t mode);
/* Column slabs of the SpMM passes (Section 4 names reordering for locality;
 * this is the blocking counterpart): a pass whose gathered block (gathered
 * rows x block width x 4 bytes) is larger than `bytes` runs as S launches over
 * column ranges of the matrix, S = ceil(block bytes / bytes) (at most 64), so
 * that the block rows one launch gathers stay in L2; each launch adds its
 * exact row sums, reduced mod p, to the output rows, the last one applies the
 * diagonal.  The slab layouts are built on first use from a copy of the CSR
 * that matrices loaded while slabs are on keep on the device (others run
 * without slabs).  0 or negative (default) = no slabs: on the
 * 1.9M x 1.95M block-32 matrix (paired block of 64 residues, 486 MB gathered
 * per pass) a pass takes 1.48 ms without slabs and 2.1-5.3 ms with 4-16 of
 * them, because every slab reads and writes all output rows.  Results never
 * depend on it. */
wr_status wr_set_column_slabs(wr_ctx *ctx, int64_t bytes);

/* ---------------------------------------------------------------- matrices */

/* Ingest a CSR matrix (Section 2.5 step 1 operates on it as a black box).
 * rowptr: rows + 1 int64, nondecreasing, rowptr[0] = 0; colidx: int32 in
 * [0, cols); vals: small signed integers (the paper's boundary matrices hold
 * 0, +-1 and small integers).  rows, cols < 2^31; every row < 2^24 entries.
 * Entries in [-127, 127] with rows, cols < 2^24 are packed with their column
 * in one 32-bit word; otherwise (entries up to |v| <= 32767, or a dimension
 * of 2^24 and more) the layout keeps 32-bit columns with int16 values beside
 * them, and every row and column must then hold fewer than 65,536 entries
 * (exact int64 sums); anything else is WR_EOVERFLOW.  Builds SELL-C-sigma
 * layouts of A and A^T on the device. */
wr_status wr_matrix_load_csr(wr_ctx *ctx, int64_t rows, int64_t cols, const int64_t *rowptr,
                             const int32_t *colidx, const int32_t *vals, wr_matrix **out);
/* Same, from arrays already in device memory (nnz = rowptr[rows]). */
wr_status wr_matrix_load_csr_device(wr_ctx *ctx, int64_t rows, int64_t cols, int64_t nnz,
                                    const int64_t *d_rowptr, const int32_t *d_colidx,
                                    const int32_t *d_vals, wr_matrix **out);
/* rows, cols, nnz, and the padded slot counts of the A and A^T layouts (of
 * the reduced matrix when the chain reduction ran). */
wr_status wr_matrix_info(const wr_matrix *mat, int64_t *rows, int64_t *cols, int64_t *nnz,
                         int64_t *slots_a, int64_t *slots_at);
void wr_matrix_free(wr_matrix *mat);

/* Chain reduction at read time (Section 2.6.4, off by default): loads through
 * this context first remove, repeatedly, every row or column whose only
 * nonzero entry is +-1, together with the column or row of that entry (a
 * free-face pair; one step of Gaussian elimination that changes nothing
 * else), and the empty rows and columns.  The matrix held is the reduced one
 * and wr_rank returns rank_offset + its rank, rank_offset being the number of
 * pivots taken.  Unit pivots are units modulo every prime, so the reduced
 * matrix serves any prime; sequences and generators are those of the reduced
 * matrix.  The reduction is a host pass (a matrix given in device memory is
 * copied to the host for it). */
wr_status wr_set_chain_reduction(wr_ctx *ctx, int32_t on);
/* Locality order at read time (off by default; the paper's conclusion names
 * an adapted reordering for clustering the products): loads through this
 * context renumber the rows and the columns by decreasing entry count, so
 * that the block rows the SpMM gathers most often sit next to each other.
 * Everything stays in the loaded order at the boundary: X, Y, D1, D2 are
 * drawn at the loaded indices, so sequences, generators and ranks are the
 * same with and without it, and the black-box calls take and return blocks
 * in the loaded row order.  A host pass (after the chain reduction, when
 * both are on). */
wr_status wr_set_locality_order(wr_ctx *ctx, int32_t on);
/* The locality order on host arrays, without a device: the renumbered CSR
 * (arrays sized as the input's) and each layout row's and column's input
 * index (rows resp. cols entries).  WR_EINVAL on a malformed CSR. */
wr_status wr_locality_order_csr(int64_t rows, int64_t cols, const int64_t *rowptr, const int32_t *colidx,
                                const int32_t *vals, int64_t *out_rowptr, int32_t *out_colidx, int32_t *out_vals,
                                int32_t *out_row_of, int32_t *out_col_of);
/* One matrix of a complex for wr_chain_reduce_complex: the input CSR (host
 * arrays, read only) and the caller's output arrays, sized as the input's
 * (rows + 1 and rowptr[rows] entries; out_row_of / out_col_of: rows / cols
 * entries, or NULL); out_rows, out_cols and rank_offset are written. */
typedef struct {
    int64_t rows, cols;
    const int64_t *rowptr;
    const int32_t *colidx;
    const int32_t *vals;
    int64_t out_rows, out_cols, rank_offset;
    int64_t *out_rowptr;
    int32_t *out_colidx, *out_vals, *out_row_of, *out_col_of;
} wr_csr_io;
/* Chain reduction along a complex (Section 2.6.4, propagation from one matrix
 * to the next), on the host.  mats[i]'s columns are mats[i+1]'s rows and
 * mats[i] mats[i+1] = 0 over Z (checked: WR_EINVAL otherwise, and on any
 * malformed CSR or size mismatch).  Every unit pivot at (r, c) of mats[i]
 * removes row r and column c there (rank_offset + 1) and, in the
 * neighbours, column r of mats[i-1] and row c of mats[i+1], lines that the
 * complex makes zero or dependent; removals cascade.  For every i and every
 * prime, rank(mats[i]) = rank_offset + rank(reduced mats[i]).  count = 1 is
 * the single-matrix reduction of wr_chain_reduce_csr. */
wr_status wr_chain_reduce_complex(int32_t count, wr_csr_io *mats);
/* The input's size and the pivots the chain reduction took (0 without it). */
wr_status wr_matrix_reduction(const wr_matrix *mat, int64_t *rows_in, int64_t *cols_in, int64_t *rank_offset);
/* The same reduction on host arrays, without a device: writes the reduced
 * CSR (rows and columns renumbered in their input order) into arrays sized
 * for the input (rows + 1 and rowptr[rows] entries) and, when the pointers
 * are not NULL, each kept row's and column's input index (rows resp. cols
 * entries at most); rank(input) = *rank_offset + rank(output) over every
 * prime field.  WR_EINVAL on a malformed CSR. */
wr_status wr_chain_reduce_csr(int64_t rows, int64_t cols, const int64_t *rowptr, const int32_t *colidx,
                              const int32_t *vals, int64_t *out_rows, int64_t *out_cols, int64_t *out_rowptr,
                              int32_t *out_colidx, int32_t *out_vals, int32_t *out_row_of, int32_t *out_col_of,
                              int64_t *rank_offset);

/* ---------------------------------------------------------------- rank */

/* Rank of the matrix modulo params->prime (Section 2.5 steps 1-4). */
wr_status wr_rank(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params, wr_result **out);

/* Many jobs in one call (matrices may repeat with different primes or seeds;
 * the paper's rank over Q takes the maximum over several primes, Section
 * 2.5).  Jobs run on the context's batch slots (wr_set_batch_slots, default
 * 8): each slot has its own stream and host thread, so the sequence loops and
 * sigma-basis kernels of several jobs are in flight on the device at once;
 * slots take the largest remaining job first.  Each job's result is
 * bit-identical to the same job run alone.  outs[j] receives job j's result
 * (NULL when that job failed; the call then returns the first failing job's
 * status, its index in wr_last_error()).  The matrices must have been loaded
 * on the context's device. */
wr_status wr_rank_batch(wr_ctx *ctx, size_t njobs, const wr_matrix *const *mats,
                        const wr_params *params, wr_result **outs);
/* Number of slots wr_rank_batch uses on this context (1..64). */
wr_status wr_set_batch_slots(wr_ctx *ctx, int32_t slots);
/* Job fusion in wr_rank_batch (on by default): jobs on the same matrix with
 * the same m = n (at most 16), side, sequence length and outputs, and any
 * primes and seeds (the rank over Q takes one matrix modulo several primes,
 * Section 2.5), run in groups of up to four sharing one sequence loop: each
 * job's X beside Y occupies a slice of one block of up to 64 columns, one
 * pair of SpMM passes per application reads the matrix once for all of them
 * (the exact int64 row sums do not depend on the prime; each slice is reduced
 * modulo its own prime and scaled by its own diagonals), the Gram
 * projections and sigma-bases run per job.  Each result is bit-identical to
 * the job run alone.  Not used with early termination. */
wr_status wr_set_batch_fusion(wr_ctx *ctx, int32_t on);
/* Upper bound of the device memory one wr_rank call on (mat, params)
 * allocates besides the loaded matrix (the server's admission estimate). */
wr_status wr_rank_device_bytes(const wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                               uint64_t *bytes);

uint64_t wr_result_rank(const wr_result *res);
/* deg det F, codeg det F = v_x(det F), sum of the generator's column degrees,
 * and the sequence length used. */
wr_status wr_result_info(const wr_result *res, int64_t *deg_det, int64_t *codeg,
                         int64_t *sum_delta, int64_t *seq_len);
/* Copy the sequence (L*m*n residues, [i][a][b]) to host memory dst (cap_elems
 * entries).  Needs WR_WANT_SEQUENCE. */
wr_status wr_result_sequence(const wr_result *res, uint32_t *dst, size_t cap_elems);
/* Copy the generator F ((dmax+1)*n*n residues, [k][row][col], dmax = max column
 * degree) and its column degrees (n).  Needs WR_WANT_GENERATOR. */
wr_status wr_result_generator(const wr_result *res, uint32_t *coeffs, size_t cap_elems,
                              int32_t *col_degrees);
void wr_result_free(wr_result *res);

/* ------------------------------------------- step-level calls (device data) */

/* One application of the preconditioned black box (Section 2.3):
 * d_out = A~ d_in, d_in, d_out: N x width residues (width 1..32), N and D1, D2
 * from params (side, seed, prime).  d_in and d_out may alias. */
wr_status wr_blackbox_apply_device(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                                   const uint32_t *d_in, uint32_t *d_out, int64_t width);
/* The same application as wr_blackbox_apply_device, without allocating any
 * device memory.  The paper has no counterpart: it exists for callers that
 * must not allocate device memory while they run -- code that works inside
 * another program's fixed device-memory arena (where cudaMalloc would fail or
 * fragment it), or latency-critical loops that cannot pay for cudaMalloc or
 * cudaFree (both may synchronise the device).  The matrix is loaded
 * beforehand with the usual calls; d_in and d_out are the caller's (N x width
 * residues each, as in wr_blackbox_apply_device).
 * Its temporaries live in one fixed 32 MiB array per device, held by every
 * device that loads the library until the process exits.  It needs
 * 4 nv (N + M) + 4 (N + M) + 8 nv (split rows of A and A^T) bytes (nv = width
 * rounded up to a power of two, M the other dimension); larger requests return
 * WR_EINVAL with the sizes in wr_last_error().  The first call on a device
 * looks up the array's device address (with that device current): make that
 * first call before any stream capture.  The address is kept per device and
 * primary context; after a device reset (cudaDeviceReset, which also ends
 * every context, matrix and stream of this library on that device) the next
 * call looks it up again.  All calls share the array and find
 * what the previous call left in it; calls whose work overlaps on the GPU
 * (other threads, contexts or streams of the same device) race on it and must
 * be serialised by the caller.  The call returns after its work completed. */
wr_status wr_blackbox_apply_device_noalloc(wr_ctx *ctx, const wr_matrix *mat,
                                           const wr_params *params, const uint32_t *d_in,
                                           uint32_t *d_out, int64_t width);
/* The sequence S_i = X^T A~^i Y, i < L (Section 2.5 step 2) into d_S (L*m*n). */
wr_status wr_sequence_device(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                             uint32_t *d_S, uint64_t L);
/* The sequence of wr_sequence_device, plus the block the iteration carries,
 * for spot checks of any step at full size (Section 2.5 step 2).  The block
 * after k applications of A~ is written in the matrix's row order, unscaled:
 * with the paired generic projection (m = n, wr_set_paired_projection) the
 * N x (m + n) block [A~^k X | A~^k Y] (*paired = 1), otherwise the N x n block
 * A~^k Y (*paired = 0).  One application yields two terms in the paired and
 * symmetric modes (S_2k = X^T A~^2k Y from the block after k applications),
 * one term otherwise.  d_snap (may be NULL) receives the block after snap_at
 * applications, d_last (may be NULL) the block after the last application;
 * *applications (may be NULL) receives the number of applications done.
 * snap_at beyond that number is WR_EINVAL. */
wr_status wr_sequence_state_device(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                                   uint32_t *d_S, uint64_t L, int64_t snap_at, uint32_t *d_snap,
                                   uint32_t *d_last, int64_t *applications, int32_t *paired);
/* One Gram projection of the sequence (Section 2.3), through the kernels the
 * sequence uses (wr_set_tensor_projection chooses them):
 * d_G (m x n) = sum_{r < N} w_r t[r][0 .. m)^T t[r][yoff .. yoff + n) mod p.
 * d_t: N rows of tstride residues (16-byte aligned; nv = n rounded up to a
 * power of two; tstride a multiple of nv with tstride >= m and >= yoff + nv;
 * yoff a multiple of nv); d_w: N residues.  All residues must be below p. */
wr_status wr_gram_device(wr_ctx *ctx, uint32_t prime, int64_t N, uint32_t m, uint32_t n, const uint32_t *d_t,
                         int32_t tstride, int32_t yoff, const uint32_t *d_w, uint32_t *d_G);
/* Columns [col0, col0 + ncols) of that sequence, S_i = X^T A~^i Y[:, col0:col0+ncols]
 * (L x m x ncols residues into d_S), with X, Y, D1, D2 drawn exactly as for
 * the whole sequence (params->n is the width of the whole Y).  The paper
 * gives every process one column of Y and gathers the column sequences before
 * the sigma-basis (Section 3.1); one GPU per column slab is the same split, and
 * the slabs of all GPUs, concatenated in column order, equal
 * wr_sequence_device's result.  With the symmetric projection X is the whole
 * Y and one term is computed per application. */
wr_status wr_sequence_slab_device(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                                  uint32_t col0, uint32_t ncols, uint32_t *d_S, uint64_t L);
/* Order-L sigma-basis of [S(x) | -I_m] with shift (0^n, 1^m) (Section 2.4):
 * writes its first n rows (the P part) as d_P ((Dcap+1) x n x (m+n), [t][r][c])
 * and the shifted column degrees d_deg (m + n).  d_S: L*m*n residues. */
wr_status wr_sigma_basis_device(wr_ctx *ctx, const uint32_t *d_S, uint64_t L, uint32_t m,
                                uint32_t n, uint32_t prime, uint32_t *d_P, int32_t *d_deg,
                                int64_t Dcap);
/* x-adic valuation of det G for G (T x n x n, [t][i][j], residues) given by
 * its first T coefficients (Section 2.5 step 4, codeg).  *val = -1 when the
 * precision T does not determine it. */
wr_status wr_det_valuation_device(wr_ctx *ctx, const uint32_t *d_G, int64_t n, int64_t T,
                                  uint32_t prime, int64_t *val);

/* The polynomial matrix product of PM-Basis (Section 2.4: the sigma-basis of
 * order L is the product of two of order L/2, and the second is computed from
 * the middle coefficients of S(x) times the first):
 * C[k - lo] = sum_j A_j B_{k-j} mod prime for lo <= k < hi (coefficients past
 * the exact product's na + nb - 2 are 0).  d_A: na coefficients of r x s,
 * d_B: nb coefficients of s x t, d_C: (hi - lo) x r x t, all device pointers
 * to residues below prime, coefficient-major and row-major inside a
 * coefficient; the caller owns every buffer.  Returns once d_C is written
 * (the context's stream is synchronised).  Computed as three number-theoretic
 * transforms over 998244353, 469762049 and 2013265921 and a Chinese remainder
 * step, so s * min(na, nb) * (prime - 1)^2 must stay below their product and
 * max(hi, na + nb - 1 - lo) at most 2^23; WR_EINVAL otherwise, and for
 * lo > hi, a negative size, r, s or t outside 1..1024, or a null pointer
 * with work to do. */
wr_status wr_polymat_mul_device(wr_ctx *ctx, uint32_t prime, const uint32_t *d_A, int64_t na,
                                const uint32_t *d_B, int64_t nb, uint32_t r, uint32_t s, uint32_t t,
                                int64_t lo, int64_t hi, uint32_t *d_C);

/* ---------------------------------------------------------------- measurement */

/* Tensor-core rate and layout probe (a measurement helper; the paper has no
 * counterpart): `blocks` thread blocks (one per SM at most) each issue
 * iters chains of four tcgen05 bf16 MMAs (M = 128, N = 256, K = 16 each, fp32
 * accumulators in tensor memory) on tiles held in shared memory; *ms is the
 * kernel's duration (CUDA events).  With d_out != NULL, block 0 writes its
 * 128 x 256 fp32 accumulator: entry (r, c) = iters * sum_{k < 64} a(r, k) b(c, k)
 * with a(r, k) = (7r + 3k) mod 17 - 8 and b(c, k) = (5c + 11k) mod 13 - 6. */
wr_status wr_probe_mma(wr_ctx *ctx, int64_t iters, int32_t blocks, float *d_out, double *ms);

/* ---------------------------------------------------------------- serving */

typedef struct {
    int32_t max_slots;        /* requests resident on the device at once                 */
    uint64_t hbm_budget;      /* bytes of device memory the admitted requests may hold   */
    int32_t queue_cap;        /* pending requests before wr_submit returns WR_EBUSY      */
} wr_server_cfg;

typedef struct {
    uint64_t submitted, completed, failed;
    double p50_ms, p99_ms;    /* latency submit -> result                                */
    double throughput_rps;    /* completed / (last completion - first submission)         */
    int32_t max_resident;     /* most requests resident at once                          */
    int64_t kernel_launches;  /* kernels launched by the server's slots so far            */
} wr_stats;

/* Continuous-batching rank server (no counterpart in the paper, which runs
 * one matrix at a time).  max_slots slots, each a stream of its own with one
 * host thread; a queued request is admitted, in arrival order, as soon as a
 * slot is idle and its device-memory estimate (wr_rank_device_bytes) fits
 * beside the requests already resident (hbm_budget; 0 = no limit; a request
 * above the budget is refused at submission with WR_EINVAL).  Requests that
 * arrive while others are on the GPU therefore start at once and overlap with
 * them on the device; each result is bit-identical to the same request run
 * alone.  Latency is measured from wr_submit to the result being ready. */
wr_status wr_server_start(wr_ctx *ctx, const wr_server_cfg *cfg, wr_server **out);
/* Queue a rank request; the matrix must stay alive until its result is taken. */
wr_status wr_submit(wr_server *srv, const wr_matrix *mat, const wr_params *params,
                    uint64_t *ticket);
/* Wait up to timeout_ms for a ticket's result (WR_ETIMEDOUT if not ready). */
wr_status wr_wait(wr_server *srv, uint64_t ticket, uint32_t timeout_ms, wr_result **out);
wr_status wr_server_stats(wr_server *srv, wr_stats *out);
void wr_server_stop(wr_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* WR_H */
