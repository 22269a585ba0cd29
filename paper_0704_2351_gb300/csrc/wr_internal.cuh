// Internal definitions shared by the CUDA translation units of libwr.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/wr.h"

namespace wr {

// ------------------------------------------------------------------ errors

void set_error(const std::string &msg);
wr_status fail(wr_status st, const std::string &msg);
wr_status cuda_fail(cudaError_t e, const char *what);

// Event flags for host waits: the waiting thread sleeps instead of spinning,
// since the pipelined and batched paths have many host threads waiting at
// once (two per job) and spinning ones would take the cores that launch work.
constexpr unsigned WAIT_EVENT_FLAGS = cudaEventBlockingSync | cudaEventDisableTiming;

// Wait, asleep, for everything queued on s so far.
inline cudaError_t sync_stream_blocking(cudaStream_t s) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, WAIT_EVENT_FLAGS);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev);
    cudaEventDestroy(ev);
    return e;
}

#define WR_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ::wr::cuda_fail(e_, #call);  \
    } while (0)

// after a kernel launch: count it on the context and check the launch
#define WR_LAUNCHED(ctx)                                                   \
    do {                                                                   \
        (ctx)->launches++;                                                 \
        cudaError_t e_ = cudaGetLastError();                               \
        if (e_ != cudaSuccess) return ::wr::cuda_fail(e_, "kernel launch"); \
    } while (0)

#define WR_TRY(call)                              \
    do {                                          \
        wr_status s_ = (call);                    \
        if (s_ != WR_OK) return s_;               \
    } while (0)

// ------------------------------------------------------------------ arithmetic mod p
//
// Residues are uint32 in [0, p), p < 2^31.  Reduction of a 64-bit value uses
// Barrett's method with mu = floor(2^64 / p): q = hi64(x * mu) is at most 2
// below floor(x / p), so r = x - q p < 3 p needs at most two corrections.
// Signed sums (|s| < 2^62) are shifted by off, a multiple of p >= 2^62.

struct ModP {
    uint32_t p;
    uint32_t lazy;   // products (p-1)^2 that fit on top of a value < p in a uint64
    uint64_t mu;     // floor(2^64 / p)
    int64_t off;     // multiple of p in [2^62, 2^62 + p)
    uint32_t pneg;   // -p^{-1} mod 2^32 (Montgomery, R = 2^32)
    uint32_t r1;     // R mod p: the Montgomery form of 1
    uint32_t r2;     // R^2 mod p
};

ModP make_modp(uint32_t p);

// Products below (p-1)^2 that fit in a 64-bit accumulator on top of what
// fold2 by c = 2^32 mod p leaves (at most c^2 + 2^32 - 1): the fold interval
// of the lazily reduced sums (at least 2 for p < 2^31, 14 for p < 2^30).
inline int fold_products(uint32_t p) {
    const unsigned __int128 c = ((unsigned __int128)1 << 32) % p;
    const unsigned __int128 after = c * c + (((unsigned __int128)1 << 32) - 1);
    const unsigned __int128 room = (((unsigned __int128)1 << 64) - 1) - after;
    const unsigned __int128 prod = (unsigned __int128)(p - 1) * (p - 1);
    return prod ? (int)std::min<unsigned __int128>(room / prod, 1000) : 1000;
}

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ uint32_t red64(uint64_t x, const ModP &m) {
    uint64_t q = mulhi64(x, m.mu);
    uint64_t r = x - q * (uint64_t)m.p;
    if (r >= m.p) r -= m.p;
    if (r >= m.p) r -= m.p;
    return (uint32_t)r;
}

#ifdef __CUDACC__
// d = a b + c in one 32x32 -> 64-bit multiply-add
__device__ __forceinline__ unsigned long long madw(uint32_t a, uint32_t b, unsigned long long c) {
    unsigned long long d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// x = hi 2^32 + lo is congruent to hi (2^32 mod p) + lo; folded twice a 64-bit
// accumulator drops to at most c^2 + 2^32 - 1 (c = 2^32 mod p), leaving room
// for fold_products(p) more products below p^2 before the next fold (at
// least 14 for p < 2^30, 2 for p < 2^31).  Two 32x32+64-bit multiply-adds
// instead of a reduction mod p.
__device__ __forceinline__ unsigned long long fold2(unsigned long long x, uint32_t c) {
    x = madw((uint32_t)(x >> 32), c, (unsigned long long)(uint32_t)x);
    return madw((uint32_t)(x >> 32), c, (unsigned long long)(uint32_t)x);
}

// A 64-bit accumulator kept as two 32-bit words: (hi, lo) += a b as two
// multiply-adds chained through the carry flag.
struct Acc2 {
    uint32_t lo, hi;
};
__device__ __forceinline__ void mac2(Acc2 &acc, uint32_t a, uint32_t b) {
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;"
        : "+r"(acc.lo), "+r"(acc.hi)
        : "r"(a), "r"(b));
}
__device__ __forceinline__ unsigned long long acc2_u64(const Acc2 &a) {
    return ((unsigned long long)a.hi << 32) | a.lo;
}
// fold2 on the two-word form
__device__ __forceinline__ void fold2w(Acc2 &a, uint32_t c) {
    const unsigned long long x = fold2(acc2_u64(a), c);
    a.lo = (uint32_t)x;
    a.hi = (uint32_t)(x >> 32);
}


#endif

__host__ __device__ __forceinline__ uint32_t red_s64(int64_t s, const ModP &m) {
    return red64((uint64_t)s + (uint64_t)m.off, m);  // |s| < 2^62: the sum is in [0, 2^64)
}

__host__ __device__ __forceinline__ uint32_t mulm(uint32_t a, uint32_t b, const ModP &m) {
    return red64((uint64_t)a * b, m);
}

__host__ __device__ __forceinline__ uint32_t addm(uint32_t a, uint32_t b, const ModP &m) {
    uint32_t s = a + b;  // < 2^32 since a, b < 2^31
    return s >= m.p ? s - m.p : s;
}

__host__ __device__ __forceinline__ uint32_t subm(uint32_t a, uint32_t b, const ModP &m) {
    return a >= b ? a - b : a + m.p - b;
}

__host__ __device__ __forceinline__ uint32_t powm(uint32_t a, uint32_t e, const ModP &m) {
    uint32_t r = 1 % m.p;
    while (e) {
        if (e & 1) r = mulm(r, a, m);
        a = mulm(a, a, m);
        e >>= 1;
    }
    return r;
}

// Montgomery product with R = 2^32: a b R^{-1} mod p for a, b < p < 2^31.
// t + m p < 2^62 + 2^63, and the result is < 2p before the correction.
__host__ __device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, const ModP &m) {
    const uint64_t t = (uint64_t)a * b;
    const uint32_t k = (uint32_t)t * m.pneg;
    const uint32_t u = (uint32_t)((t + (uint64_t)k * m.p) >> 32);
    return u >= m.p ? u - m.p : u;
}

// Montgomery reduction of a 64-bit T < p 2^32: T R^{-1} mod p.
__host__ __device__ __forceinline__ uint32_t mont_redc(uint64_t t, const ModP &m) {
    const uint32_t k = (uint32_t)t * m.pneg;
    const uint32_t u = (uint32_t)((t + (uint64_t)k * m.p) >> 32);
    return u >= m.p ? u - m.p : u;
}

__host__ __device__ __forceinline__ uint32_t to_mont(uint32_t a, const ModP &m) { return mont_mul(a, m.r2, m); }
__host__ __device__ __forceinline__ uint32_t from_mont(uint32_t a, const ModP &m) { return mont_mul(a, 1u, m); }

// (a R)^{-1} R = a^{-1} R in Montgomery form, by Fermat's little theorem
__host__ __device__ __forceinline__ uint32_t mont_inv(uint32_t am, const ModP &m) {
    uint32_t r = m.r1, b = am, e = m.p - 2;
    while (e) {
        if (e & 1) r = mont_mul(r, b, m);
        b = mont_mul(b, b, m);
        e >>= 1;
    }
    return r;
}

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// inverse of a != 0 by Fermat's little theorem
__host__ __device__ __forceinline__ uint32_t invm(uint32_t a, const ModP &m) {
    return powm(a, m.p - 2, m);
}

// ------------------------------------------------------------------ random draws
//
// SplitMix64 (Steele, Lea, Flood 2014): output for state x is the mix of
// x + 0x9E3779B97F4A7C15.  Entry idx of the stream with tag t under seed s is
// h = sm(sm(s ^ t * GOLDEN) + idx).

constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ULL;

__host__ __device__ __forceinline__ uint64_t sm64(uint64_t x) {
    uint64_t z = x + GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t stream_hash(uint64_t seed, uint64_t tag, uint64_t idx) {
    return sm64(sm64(seed ^ (tag * GOLDEN)) + idx);
}

enum { TAG_X = 1, TAG_Y = 2, TAG_D1 = 3, TAG_D2 = 4 };

bool is_prime_u32(uint64_t n);

// ------------------------------------------------------------------ device memory

// Device allocation in stream order on the context's stream
// (cudaMallocAsync / cudaFreeAsync): a buffer released at scope exit is
// freed after the work already queued on that stream.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    wr_free_fn free_fn = nullptr;  // caller's allocator (nullptr: cudaFreeAsync)
    void *free_user = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept
        : ptr(o.ptr), bytes(o.bytes), stream(o.stream), free_fn(o.free_fn), free_user(o.free_user) {
        o.ptr = nullptr;
        o.bytes = 0;
    }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            ptr = o.ptr; bytes = o.bytes; stream = o.stream; free_fn = o.free_fn; free_user = o.free_user;
            o.ptr = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void release();
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// ------------------------------------------------------------------ sparse layout
//
// Two parts per matrix (one for A, one for A^T):
//  * SELL-C-sigma part for light rows (at most LIGHT_MAX entries, empty rows
//    included): rows sorted by length (descending), packed by chunks of 32,
//    slot-major: entry j of lane r of chunk c is at entries[off[c] + 32 j + r],
//    a packed word (col << 8) | (uint8)val; padding words are 0.  vrow[32 c + r]
//    is the output row, or EMPTY past the last light row.
//  * vector part for longer rows: entries copied contiguously (ventries) and
//    cut into segments of at most VSEG entries, one warp per segment.
//    seg_row is the output row, or SPLIT | split_id for rows with more than one
//    segment: those add exact int64 partial sums into an accumulator that a
//    second kernel reduces, scales and stores.

constexpr int SELL_C = 32;
constexpr int LIGHT_MAX = 64;
constexpr int VSEG = 256;
constexpr uint32_t VROW_SPLIT = 0x80000000u;
constexpr uint32_t VROW_EMPTY = 0xFFFFFFFFu;

struct Sell {
    int64_t nrows = 0;     // output rows
    int64_t ncols = 0;     // gathered dimension
    // light part
    int64_t nlight = 0;
    int64_t nchunks = 0;
    int64_t nslots = 0;    // entries incl. padding
    DevBuf entries;        // uint32 [nslots]
    DevBuf chunk_off;      // int64  [nchunks + 1]
    DevBuf chunk_len;      // int32  [nchunks]
    DevBuf vrow;           // uint32 [nchunks * 32]
    // vector part
    int64_t nseg = 0;
    int64_t nvent = 0;
    DevBuf ventries;       // uint32 [nvent]
    DevBuf seg_start;      // int64  [nseg]
    DevBuf seg_len;        // int32  [nseg]
    DevBuf seg_row;        // uint32 [nseg]
    int64_t nsplit = 0;    // rows with more than one segment
    DevBuf split_row;      // int32  [nsplit]
    // wide layout (entries outside [-127, 127] or a dimension >= 2^24): the
    // entry words hold the column alone and the values sit beside them
    bool wide = false;
    DevBuf wvals;          // int16  [nslots]
    DevBuf vwvals;         // int16  [nvent]
};

struct SellView {
    int64_t nrows, ncols, nchunks, nseg, nsplit;
    const uint32_t *entries;
    const int64_t *chunk_off;
    const int32_t *chunk_len;
    const uint32_t *vrow;
    const uint32_t *ventries;
    const int64_t *seg_start;
    const int32_t *seg_len;
    const uint32_t *seg_row;
    const int32_t *split_row;
    const int16_t *wvals;   // wide layout only
    const int16_t *vwvals;
};

inline SellView view(const Sell &s) {
    return SellView{s.nrows, s.ncols, s.nchunks, s.nseg, s.nsplit, s.entries.as<uint32_t>(),
                    s.chunk_off.as<int64_t>(), s.chunk_len.as<int32_t>(), s.vrow.as<uint32_t>(),
                    s.ventries.as<uint32_t>(), s.seg_start.as<int64_t>(), s.seg_len.as<int32_t>(),
                    s.seg_row.as<uint32_t>(), s.split_row.as<int32_t>(),
                    s.wide ? s.wvals.as<int16_t>() : nullptr, s.wide ? s.vwvals.as<int16_t>() : nullptr};
}

}  // namespace wr

// ------------------------------------------------------------------ opaque handles

namespace wr {
// Terms of a sequence that one host thread computes while another consumes
// them: once ev[i] has completed on the producer's stream, S_0 .. S_{ready[i]-1}
// are final in the device sequence buffer.  The owner destroys the events.
struct SeqFeed {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<cudaEvent_t> ev;
    std::vector<int64_t> ready;
    bool closed = false;    // the producer has recorded its last event (or stopped)
    int64_t waited = -1;    // consumer: last event index its stream waits on
    // early termination: the producer keeps at most `throttle` groups in
    // flight (0: no limit) and stops once it has published stop_at terms;
    // the consumer sets orders_used to the orders its sigma-basis took
    int throttle = 0;
    std::atomic<int64_t> stop_at{INT64_MAX};
    int64_t orders_used = -1;
};
}  // namespace wr

struct wr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    size_t smem_optin = 0;
    bool profiling = false;
    int64_t launches = 0;   // kernels launched through this context (graph replays: nodes per replay)
    int batch_slots = 8;    // slots (streams + host threads) of wr_rank_batch
    bool batch_fuse = true; // wr_rank_batch: jobs on one matrix share one sequence loop
    int sigma_chunk = 0;    // orders per sigma-basis chunk (0: automatic)
    int64_t sigma_leaf = 0; // orders per PM-Basis leaf (0: automatic)
    bool autotune = true;   // tune the SpMM lane width per matrix and block width
    int lane_width = 0;     // forced SpMM residues per lane (0: tuned or default)
    bool pair_generic = true; // generic projection, m = n: X and Y in one block, two terms per application
    int tensor_proj = -1;   // Gram projections on the tensor cores: 1 on, 0 off, -1 automatic
    bool proj_overlap = false; // Gram projections on a side stream beside the SpMM passes
    int pipeline = 1;       // wr_rank: the sigma-basis trails the sequence on a second stream
                            // (0 off, 1 automatic priority, 2 the sigma-basis's stream first,
                            // 3 the sequence's first)
    bool high_priority = false; // this context's own stream has the greatest priority
    bool seq_high = false;      // seq_stream has the greatest priority
    int64_t early_term = 0; // quiet orders that end the sequence early (0: the full L terms)
    bool chain_reduce = false; // matrix loads: remove unit singleton rows/columns and empty ones
    bool reorder = false;      // matrix loads: renumber rows and columns by decreasing degree
    int64_t slab_bytes = 0;    // column slabs: gathered block bytes per slab (<= 0: off)
    wr_ctx *aux = nullptr;  // child context (own stream) that runs the trailing sigma-basis
    cudaStream_t seq_stream = nullptr; // high-priority stream of the pipelined sequence (lazy)
    wr::SeqFeed *feed = nullptr; // set on a child context while it consumes a sequence in flight
    wr_alloc_fn alloc_fn = nullptr;  // caller's device allocator (nullptr: cudaMallocAsync)
    wr_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    wr_timings last{};
    // PM-Basis products: twiddle tables of the transform primes for lengths
    // up to 2^ntt_lg (0: none yet), released before the stream
    wr::DevBuf ntt_tw;
    int ntt_lg = 0;
};

struct wr_matrix {
    wr_ctx *ctx = nullptr;
    int64_t rows = 0, cols = 0, nnz = 0;
    // chain reduction at load: the matrix held is the reduced one, of the
    // rows_in x cols_in input; rank(input) = rank_offset + rank(held)
    int64_t rows_in = 0, cols_in = 0, rank_offset = 0;
    // locality order: layout row i is row map_rows[i] of the matrix as
    // loaded (after any chain reduction), column j is column map_cols[j];
    // empty when the matrix keeps its order
    wr::DevBuf map_rows, map_cols;
    wr::Sell a;    // rows of A
    wr::Sell at;   // rows of A^T
    bool wide = false;
    // the CSR of A ([0]) and of A^T ([1]), kept on the device for column slabs
    wr::DevBuf csr_rp[2], csr_ci[2], csr_va[2];
    // column-slab layouts of A ([0]) and A^T ([1]), built on first use for the
    // slab count in slab_n (the last one asked for)
    mutable std::vector<wr::Sell> slabs[2];
    mutable int slab_n[2] = {0, 0};
    // SpMM residues per lane tuned for [layout a / at][log2 block width] (0: not yet)
    mutable std::mutex tune_mu;
    mutable int tuned_w[2][7] = {{0}};
};

struct wr_result {
    uint32_t prime = 0, m = 0, n = 0;
    int64_t rank = 0, deg_det = 0, codeg = 0, sum_delta = 0, seq_len = 0;
    std::vector<uint32_t> seq;       // L*m*n (when wanted)
    std::vector<uint32_t> gen;       // (dmax+1)*n*n (when wanted)
    std::vector<int32_t> gen_deg;    // n
    int64_t gen_dmax = -1;
};

namespace wr {

wr_status dev_alloc(wr_ctx *ctx, DevBuf &b, size_t bytes);

// chain reduction (wr_reduce.cu): the reduced CSR, its rows' and columns'
// indices in the input, and the number of unit pivots taken
struct ReducedCsr {
    int64_t rows = 0, cols = 0, rows_in = 0, cols_in = 0, rank_offset = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colidx, vals, row_of, col_of;
};
wr_status chain_reduce_host(int64_t rows, int64_t cols, const int64_t *rowptr, const int32_t *colidx,
                            const int32_t *vals, ReducedCsr &out);
wr_status chain_reduce_complex_host(int count, wr_csr_io *io);
// Locality order (wr_reduce.cu): rows and columns renumbered by decreasing
// entry count (ties by index); out.row_of / col_of map back, rank_offset = 0.
wr_status locality_order_host(int64_t rows, int64_t cols, const int64_t *rowptr, const int32_t *colidx,
                              const int32_t *vals, ReducedCsr &out);

// format (wr_format.cu)
wr_status build_sell(wr_ctx *ctx, int64_t rows, int64_t cols, int64_t nnz, const int64_t *d_rowptr,
                     const int32_t *d_colidx, const int32_t *d_vals, Sell &out, bool wide);
wr_status build_sell_slab(wr_ctx *ctx, int64_t rows, int64_t cols, const int64_t *d_rowptr, const int32_t *d_colidx,
                          const int32_t *d_vals, int32_t c0, int32_t c1, Sell &out, bool wide);
wr_status transpose_csr(wr_ctx *ctx, int64_t rows, int64_t cols, int64_t nnz, const int64_t *d_rowptr,
                        const int32_t *d_colidx, const int32_t *d_vals, DevBuf &rowptr_t,
                        DevBuf &colidx_t, DevBuf &vals_t);
wr_status validate_csr(wr_ctx *ctx, int64_t rows, int64_t cols, int64_t nnz, const int64_t *d_rowptr,
                       const int32_t *d_colidx, const int32_t *d_vals, bool *wide);
wr_status exclusive_scan_i64(wr_ctx *ctx, const int64_t *d_in, int64_t *d_out, int64_t n);

// Several jobs on one matrix in one SpMM pass (wr_multi.cu): the block holds
// `jobs` slices of 2^jw_log columns side by side, slice g reduced modulo
// mp[g] and scaled by scale[g] in the epilogue (the exact int64 row sums do
// not depend on the prime).
constexpr int MULTI_MAX_JOBS = 4;
struct MultiEpi {
    int jobs = 1;
    int jw_log = 0;
    ModP mp[MULTI_MAX_JOBS];
    const uint32_t *scale[MULTI_MAX_JOBS] = {nullptr, nullptr, nullptr, nullptr};
};

// sequence (wr_spmm.cu)
// Optional exports of the iterated block (the matrix's row order, unscaled:
// [A~^k X | A~^k Y] with the paired block, A~^k Y otherwise): after `snap_at`
// applications into d_snap, after the last one into d_last (either may be null).
struct StateOut {
    int64_t snap_at = -1;
    uint32_t *d_snap = nullptr;
    uint32_t *d_last = nullptr;
    int64_t applications = 0;  // written: applications done
    bool paired = false;       // written: whether the block carried X beside Y
};
wr_status polymat_mul(wr_ctx *ctx, const uint32_t *A, int64_t na, const uint32_t *B, int64_t nb, int r, int s,
                      int t, int64_t lo, int64_t hi, uint32_t p, uint32_t *C);
wr_status run_sequence(wr_ctx *ctx, const wr_matrix *mat, const wr_params &prm, int64_t L,
                       uint32_t *d_S, double *setup_ms, double *seq_ms, SeqFeed *feed = nullptr,
                       StateOut *out = nullptr);
// Make the context's stream wait until S_0 .. S_{terms-1} of the fed sequence
// are final (blocks the host until the producer has recorded that far).
wr_status feed_wait(wr_ctx *ctx, SeqFeed *feed, int64_t terms);
// A context on the parent's device with its own stream and the parent's settings.
// A context on the parent's device with the parent's settings and a stream
// of its own, of the greatest priority when high (else the least).
wr_status make_child(const wr_ctx *parent, wr_ctx **out, bool high = false);
// Whether sigma_basis, trailing a sequence of L terms with blocks m x n,
// runs PM-Basis in segments (else the blocked M-Basis chunk by chunk).
bool sigma_pm_trailing(const wr_ctx *ctx, int64_t L, int m, int n);
// Whether sigma_basis runs PM-Basis for L orders (else the blocked M-Basis;
// early: early termination asked for, which needs the M-Basis).
bool sigma_uses_pm(const wr_ctx *ctx, int64_t L, int m, int n, bool early = false);
void copy_settings(const wr_ctx *parent, wr_ctx *child);
wr_status blackbox_apply(wr_ctx *ctx, const wr_matrix *mat, const wr_params &prm,
                         const uint32_t *d_in, uint32_t *d_out, int64_t width);
// tensor-core Gram products (wr_gram_tc.cu): S_raw[k] += sum_r w_r t[r][0..m)^T
// t[r][yoff..yoff+n) mod p, w in Montgomery form, k = tmul * counter + toff
bool gram_tc_supported(int m, int n, int tstride, int yoff);
wr_status launch_gram_tc(wr_ctx *ctx, int64_t N, int m, int n, const uint32_t *w, const uint32_t *t, int tstride,
                         int yoff, unsigned long long *s_raw, const int *term_counter, int tmul, int toff, int64_t L,
                         const ModP &mp, int *err);
wr_status probe_mma(wr_ctx *ctx, int64_t iters, int blocks, float *d_out, double *ms);
wr_status gram_device(wr_ctx *ctx, uint32_t p, int64_t N, int m, int n, const uint32_t *t, int tstride, int yoff,
                      const uint32_t *w, uint32_t *G);
// one SpMM pass of a multi-job block (nv = the whole block width; variant as
// for the sequence: lane width, optionally | 16 for the streaming hints)
wr_status launch_spmm_multi(wr_ctx *ctx, int nv, const SellView &A, const uint32_t *x, uint32_t *y,
                            unsigned long long *acc64, const MultiEpi &me, int *term_counter, int variant);
wr_status spmm_variant_for(wr_ctx *ctx, const wr_matrix *mat, const Sell &S, int nv, int *out);
wr_status blackbox_apply_noalloc(wr_ctx *ctx, const wr_matrix *mat, const wr_params &prm,
                                 const uint32_t *d_in, uint32_t *d_out, int64_t width);

// sigma-basis and readout (wr_sigma.cu)
wr_status sigma_basis(wr_ctx *ctx, const uint32_t *d_S, int64_t L, int m, int n, uint32_t p,
                      uint32_t *d_P, int32_t *d_deg, int64_t Dcap);
wr_status det_valuation(wr_ctx *ctx, const uint32_t *d_G, int64_t n, int64_t T, uint32_t p,
                        int64_t *val);
struct Readout {
    int64_t rank, deg_det, codeg, sum_delta, vP, dmax;
    std::vector<int32_t> delta;
};
wr_status rank_readout(wr_ctx *ctx, const uint32_t *d_P, const int32_t *d_deg, int m, int n,
                       uint32_t p, int64_t Dcap, Readout &out, std::vector<uint32_t> *gen);

// parameters
struct Resolved {
    uint32_t p;
    int m, n;            // block sizes
    int nv;              // padded block width (1, 2, 4, 8, 16, 32)
    int side;            // 0: N = cols, 1: N = rows
    int64_t N, M;        // dimension of A~ and the other dimension
    int64_t L;
    bool symmetric;
    uint64_t seed;
    // the columns of Y this run carries: entry (i, b) of the block is
    // Y[i][ycol0 + b] of a Y with ystride columns (a column slab when
    // ycol0 > 0 or n < ystride); X entry (i, a) draws tag xtag at i*xwidth + a
    int ystride, ycol0;
    uint64_t xtag;
    int xwidth;
    bool gram;  // two terms per application (symmetric projection, whole Y)
    // generic projection with m = n: [D1 X | D1 Y] ride side by side, two
    // terms per application (cross Gram products); nvs = the SpMM width
    bool paired = false;
    int nvs = 0;
    // locality-ordered matrix: loaded-order index of each layout row of the
    // N-space and of the other space (nullptr: identity)
    const uint32_t *nmap = nullptr, *mmap = nullptr;
};
wr_status resolve(const wr_matrix *mat, const wr_params *prm, Resolved &r);

wr_status run_sequence_resolved(wr_ctx *ctx, const wr_matrix *mat, Resolved r, int64_t L, uint32_t *d_S,
                                double *setup_ms, double *seq_ms, SeqFeed *feed = nullptr, StateOut *out = nullptr);
// whether the generic projection pairs X with Y in one block (m = n)
bool pairs_generic(const wr_ctx *ctx, const Resolved &r);

int padded_width(int n);
bool multi_eligible(const wr_ctx *ctx, const Resolved &r);
int multi_max_jobs(const Resolved &r);
// the sequences of 1..4 jobs on one matrix in one loop (same m = n, side, L)
struct SeqFeed;
wr_status run_sequence_multi(wr_ctx *ctx, const wr_matrix *mat, const std::vector<Resolved> &rs,
                             const std::vector<uint32_t *> &d_S, double *seq_ms,
                             const std::vector<SeqFeed *> *feeds = nullptr);

}  // namespace wr
