// The C ABI of libwr (include/wr.h): contexts, matrices, the rank call,
// results and the step-level calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "wr_internal.cuh"

namespace wr {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

wr_status fail(wr_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

wr_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return WR_EDEVICE;
}

void DevBuf::release() {
    if (ptr) {
        if (free_fn) free_fn(ptr, bytes, (void *)stream, free_user);
        else cudaFreeAsync(ptr, stream);
    }
    ptr = nullptr;
    bytes = 0;
}

// Device buffers come from the caller's allocator when one is set
// (wr_set_allocator), else from the stream-ordered pool (cudaMallocAsync);
// either way they are used on ctx->stream only and returned on it.
wr_status dev_alloc(wr_ctx *ctx, DevBuf &b, size_t bytes) {
    b.release();
    if (bytes == 0) bytes = 1;
    void *p = nullptr;
    if (ctx->alloc_fn) {
        p = ctx->alloc_fn(bytes, (void *)ctx->stream, ctx->alloc_user);
        if (!p) return fail(WR_ENOMEM, "the caller's allocator returned no memory for " + std::to_string(bytes) + " bytes");
        b.free_fn = ctx->free_fn;
        b.free_user = ctx->alloc_user;
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(WR_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                       " bytes failed: " + cudaGetErrorString(e));
        }
        b.free_fn = nullptr;
        b.free_user = nullptr;
    }
    b.ptr = p;
    b.bytes = bytes;
    b.stream = ctx->stream;
    return WR_OK;
}

ModP make_modp(uint32_t p) {
    ModP m;
    m.p = p;
    m.mu = (uint64_t)(((unsigned __int128)1 << 64) / p);
    uint64_t k = ((uint64_t(1) << 62) + p - 1) / p;
    m.off = (int64_t)(k * (uint64_t)p);
    uint64_t pm1 = (uint64_t)p - 1;
    unsigned __int128 room = ((unsigned __int128)1 << 64) - 1 - p;
    uint64_t lazy = pm1 ? (uint64_t)(room / ((unsigned __int128)pm1 * pm1)) : 1024;
    m.lazy = (uint32_t)std::min<uint64_t>(lazy, 1024);
    uint32_t inv = p;  // Newton iteration for p^{-1} mod 2^32 (p odd)
    for (int i = 0; i < 5; i++) inv *= 2u - p * inv;
    m.pneg = 0u - inv;
    m.r1 = (uint32_t)((uint64_t(1) << 32) % p);
    m.r2 = (uint32_t)((uint64_t)m.r1 * m.r1 % p);
    return m;
}

static uint64_t host_powmod(uint64_t a, uint64_t e, uint64_t n) {
    unsigned __int128 r = 1 % n, b = a % n;
    while (e) {
        if (e & 1) r = r * b % n;
        b = b * b % n;
        e >>= 1;
    }
    return (uint64_t)r;
}

// deterministic Miller-Rabin for n < 2^32 (bases 2, 7, 61)
bool is_prime_u32(uint64_t n) {
    if (n < 2) return false;
    for (uint64_t sp : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull}) {
        if (n == sp) return true;
        if (n % sp == 0) return false;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (uint64_t a : {2ull, 7ull, 61ull}) {
        uint64_t x = host_powmod(a % n, d, n);
        if (a % n == 0 || x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; r++) {
            x = (uint64_t)((unsigned __int128)x * x % n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

int padded_width(int n) {
    int nv = 1;
    while (nv < n) nv <<= 1;
    return nv;
}

wr_status resolve(const wr_matrix *mat, const wr_params *prm, Resolved &r) {
    if (!mat || !prm) return fail(WR_EINVAL, "null matrix or params");
    if (prm->prime <= 2 || prm->prime >= (1u << 31) || !is_prime_u32(prm->prime))
        return fail(WR_ENOTPRIME, "prime must be a prime p with 2 < p < 2^31");
    if (prm->m < 1 || prm->m > 32 || prm->n < 1 || prm->n > 32)
        return fail(WR_EINVAL, "block sizes m, n must be in 1..32");
    if (prm->projection != WR_PROJ_GENERIC && prm->projection != WR_PROJ_SYMMETRIC)
        return fail(WR_EINVAL, "unknown projection mode");
    if (prm->projection == WR_PROJ_SYMMETRIC && prm->m != prm->n)
        return fail(WR_EINVAL, "the symmetric projection needs m = n");
    r.p = prm->prime;
    r.m = (int)prm->m;
    r.n = (int)prm->n;
    r.nv = padded_width(r.n);
    int side = prm->side;
    if (side == WR_SIDE_AUTO) side = mat->rows >= mat->cols ? WR_SIDE_COLS : WR_SIDE_ROWS;
    if (side != WR_SIDE_COLS && side != WR_SIDE_ROWS) return fail(WR_EINVAL, "unknown side");
    r.side = side;
    r.N = side == WR_SIDE_COLS ? mat->cols : mat->rows;
    r.M = side == WR_SIDE_COLS ? mat->rows : mat->cols;
    r.L = prm->seq_len ? (int64_t)prm->seq_len : (r.N + r.m - 1) / r.m + (r.N + r.n - 1) / r.n + 2;
    r.symmetric = prm->projection == WR_PROJ_SYMMETRIC;
    r.seed = prm->seed;
    r.ystride = r.n;
    r.ycol0 = 0;
    r.xtag = r.symmetric ? TAG_Y : TAG_X;
    r.xwidth = r.symmetric ? r.n : r.m;
    r.gram = r.symmetric;
    r.paired = false;
    r.nvs = r.nv;
    const uint32_t *mr = mat->map_rows.ptr ? mat->map_rows.as<uint32_t>() : nullptr;
    const uint32_t *mc = mat->map_cols.ptr ? mat->map_cols.as<uint32_t>() : nullptr;
    r.nmap = side == WR_SIDE_COLS ? mc : mr;
    r.mmap = side == WR_SIDE_COLS ? mr : mc;
    return WR_OK;
}

}  // namespace wr

using namespace wr;

// ------------------------------------------------------------------ context

extern "C" wr_status wr_create(wr_ctx **out, int device, void *cuda_stream) {
    if (!out) return fail(WR_EINVAL, "null output pointer");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(WR_EDEVICE, "no CUDA device available");
    }
    if (device < 0 || device >= ndev) return fail(WR_EINVAL, "device index out of range");
    WR_CUDA(cudaSetDevice(device));
    wr_ctx *c = new wr_ctx();
    c->device = device;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaStreamCreate"); }
        c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)optin;
    *out = c;
    return WR_OK;
}

extern "C" void wr_destroy(wr_ctx *ctx) {
    if (!ctx) return;
    if (ctx->aux) wr_destroy(ctx->aux);
    cudaSetDevice(ctx->device);
    if (ctx->seq_stream) {
        cudaStreamSynchronize(ctx->seq_stream);
        cudaStreamDestroy(ctx->seq_stream);
    }
    cudaStreamSynchronize(ctx->stream);
    ctx->ntt_tw.release();
    cudaStreamSynchronize(ctx->stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

extern "C" const char *wr_last_error(void) { return g_err.c_str(); }

extern "C" wr_status wr_set_profiling(wr_ctx *ctx, int on) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    ctx->profiling = on != 0;
    return WR_OK;
}

extern "C" wr_status wr_set_sigma_chunk(wr_ctx *ctx, int32_t orders) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    if (orders < 0 || orders > 64) return fail(WR_EINVAL, "sigma-basis chunk must be in 0..64 (0: automatic)");
    ctx->sigma_chunk = orders;
    return WR_OK;
}

extern "C" wr_status wr_set_sigma_leaf(wr_ctx *ctx, int64_t orders) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    if (orders != 0 && orders < 64) return fail(WR_EINVAL, "PM-Basis leaf must be 0 (automatic) or at least 64 orders");
    ctx->sigma_leaf = orders;
    return WR_OK;
}

extern "C" wr_status wr_set_allocator(wr_ctx *ctx, wr_alloc_fn alloc, wr_free_fn release, void *user) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    if ((alloc == nullptr) != (release == nullptr)) return fail(WR_EINVAL, "give both allocator callbacks or neither");
    ctx->alloc_fn = alloc;
    ctx->free_fn = release;
    ctx->alloc_user = user;
    return WR_OK;
}

extern "C" wr_status wr_set_autotune(wr_ctx *ctx, int32_t on) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    ctx->autotune = on != 0;
    return WR_OK;
}

extern "C" wr_status wr_set_lane_width(wr_ctx *ctx, int32_t residues) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    const int w = residues & 15;
    if ((residues & ~31) != 0 || (residues != 0 && w != 1 && w != 2 && w != 4 && w != 8))
        return fail(WR_EINVAL, "lane width must be 0 (tuned or default) or 1, 2, 4 or 8 residues, plus 16 for the "
                               "streaming cache hints");
    ctx->lane_width = residues;
    return WR_OK;
}

extern "C" wr_status wr_set_early_termination(wr_ctx *ctx, int64_t orders) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    if (orders < 0) return fail(WR_EINVAL, "early termination: orders must be >= 0 (0: off)");
    ctx->early_term = orders;
    return WR_OK;
}

extern "C" wr_status wr_set_pipeline(wr_ctx *ctx, int32_t mode) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    if (mode < 0 || mode > 3)
        return fail(WR_EINVAL, "pipeline mode must be 0 (off), 1 (automatic), 2 (sigma-basis first) or 3 (sequence first)");
    ctx->pipeline = mode;
    return WR_OK;
}

extern "C" wr_status wr_set_projection_overlap(wr_ctx *ctx, int32_t on) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    ctx->proj_overlap = on != 0;
    return WR_OK;
}

extern "C" wr_status wr_set_paired_projection(wr_ctx *ctx, int32_t on) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    ctx->pair_generic = on != 0;
    return WR_OK;
}

extern "C" wr_status wr_set_column_slabs(wr_ctx *ctx, int64_t bytes) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    ctx->slab_bytes = bytes;
    return WR_OK;
}

extern "C" wr_status wr_set_tensor_projection(wr_ctx *ctx, int32_t mode) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    if (mode < -1 || mode > 1) return fail(WR_EINVAL, "tensor projection mode must be -1 (automatic), 0 or 1");
    ctx->tensor_proj = mode;
    return WR_OK;
}

extern "C" wr_status wr_last_timings(const wr_ctx *ctx, wr_timings *out) {
    if (!ctx || !out) return fail(WR_EINVAL, "null argument");
    *out = ctx->last;
    out->kernel_launches = ctx->launches;
    return WR_OK;
}

// ------------------------------------------------------------------ matrices

static wr_status load_device(wr_ctx *ctx, int64_t rows, int64_t cols, int64_t nnz, const int64_t *d_rowptr,
                             const int32_t *d_colidx, const int32_t *d_vals, wr_matrix **out) {
    if (!ctx || !out) return fail(WR_EINVAL, "null argument");
    *out = nullptr;
    if (rows < 0 || cols < 0 || nnz < 0) return fail(WR_EINVAL, "negative size");
    if (rows >= (int64_t(1) << 31) || cols >= (int64_t(1) << 31))
        return fail(WR_EOVERFLOW, "rows and cols must be < 2^31");
    if (nnz > 0 && (!d_colidx || !d_vals)) return fail(WR_EINVAL, "null column or value array");
    if (!d_rowptr) return fail(WR_EINVAL, "null row pointer array");
    WR_CUDA(cudaSetDevice(ctx->device));
    bool wide = rows >= (int64_t(1) << 24) || cols >= (int64_t(1) << 24);
    WR_TRY(validate_csr(ctx, rows, cols, nnz, d_rowptr, d_colidx, d_vals, &wide));
    wr_matrix *m = new wr_matrix();
    m->ctx = ctx;
    m->rows = rows;
    m->cols = cols;
    m->nnz = nnz;
    m->wide = wide;
    wr_status st = build_sell(ctx, rows, cols, nnz, d_rowptr, d_colidx, d_vals, m->a, wide);
    if (st == WR_OK) {
        DevBuf rpt, cit, vat;
        st = transpose_csr(ctx, rows, cols, nnz, d_rowptr, d_colidx, d_vals, rpt, cit, vat);
        if (st == WR_OK && wide) {  // column lengths: the rows of A^T
            bool w2 = true;
            st = validate_csr(ctx, cols, rows, nnz, rpt.as<int64_t>(), cit.as<int32_t>(), vat.as<int32_t>(), &w2);
        }
        if (st == WR_OK)
            st = build_sell(ctx, cols, rows, nnz, rpt.as<int64_t>(), cit.as<int32_t>(), vat.as<int32_t>(), m->at,
                            wide);
        // with column slabs on, both CSRs stay on the device for the slab
        // layouts built on first use
        const bool keep = ctx->slab_bytes > 0;
        if (st == WR_OK && keep) st = dev_alloc(ctx, m->csr_rp[0], sizeof(int64_t) * (rows + 1));
        if (st == WR_OK && keep) st = dev_alloc(ctx, m->csr_ci[0], sizeof(int32_t) * std::max<int64_t>(nnz, 1));
        if (st == WR_OK && keep) st = dev_alloc(ctx, m->csr_va[0], sizeof(int32_t) * std::max<int64_t>(nnz, 1));
        if (st == WR_OK && keep) {
            cudaError_t e = cudaMemcpyAsync(m->csr_rp[0].ptr, d_rowptr, sizeof(int64_t) * (rows + 1),
                                            cudaMemcpyDeviceToDevice, ctx->stream);
            if (e == cudaSuccess && nnz > 0)
                e = cudaMemcpyAsync(m->csr_ci[0].ptr, d_colidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice,
                                    ctx->stream);
            if (e == cudaSuccess && nnz > 0)
                e = cudaMemcpyAsync(m->csr_va[0].ptr, d_vals, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice,
                                    ctx->stream);
            if (e != cudaSuccess) st = cuda_fail(e, "keep CSR");
        }
        if (st == WR_OK && keep) {
            m->csr_rp[1] = std::move(rpt);
            m->csr_ci[1] = std::move(cit);
            m->csr_va[1] = std::move(vat);
        }
    }
    if (st != WR_OK) {
        delete m;
        return st;
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "matrix build");
    }
    *out = m;
    return WR_OK;
}

static wr_status load_host_plain(wr_ctx *ctx, int64_t rows, int64_t cols, const int64_t *rowptr,
                                 const int32_t *colidx, const int32_t *vals, wr_matrix **out);

static wr_status upload_map(wr_ctx *ctx, const std::vector<int32_t> &m, DevBuf &dst) {
    WR_TRY(dev_alloc(ctx, dst, sizeof(uint32_t) * std::max<size_t>(m.size(), 1)));
    if (!m.empty())
        WR_CUDA(cudaMemcpyAsync(dst.ptr, m.data(), sizeof(uint32_t) * m.size(), cudaMemcpyHostToDevice, ctx->stream));
    WR_CUDA(cudaStreamSynchronize(ctx->stream));
    return WR_OK;
}

// Read-time passes on the host: the chain reduction, then the locality
// order; the matrix held is the result, with the reduction's rank offset and
// the order's index maps.
static wr_status load_prepared(wr_ctx *ctx, int64_t rows, int64_t cols, const int64_t *rowptr,
                               const int32_t *colidx, const int32_t *vals, wr_matrix **out) {
    ReducedCsr red, ord;
    int64_t R = rows, C = cols, off = 0;
    const int64_t *rp = rowptr;
    const int32_t *ci = colidx, *va = vals;
    if (ctx->chain_reduce) {
        WR_TRY(chain_reduce_host(rows, cols, rowptr, colidx, vals, red));
        R = red.rows, C = red.cols, off = red.rank_offset;
        rp = red.rowptr.data(), ci = red.colidx.data(), va = red.vals.data();
    }
    if (ctx->reorder) {
        WR_TRY(locality_order_host(R, C, rp, ci, va, ord));
        rp = ord.rowptr.data(), ci = ord.colidx.data(), va = ord.vals.data();
    }
    WR_TRY(load_host_plain(ctx, R, C, rp, ci, va, out));
    wr_matrix *m = *out;
    m->rows_in = rows;
    m->cols_in = cols;
    m->rank_offset = off;
    wr_status st = WR_OK;
    if (ctx->reorder) {
        st = upload_map(ctx, ord.row_of, m->map_rows);
        if (st == WR_OK) st = upload_map(ctx, ord.col_of, m->map_cols);
    }
    if (st != WR_OK) {
        delete m;
        *out = nullptr;
    }
    return st;
}

extern "C" wr_status wr_matrix_load_csr_device(wr_ctx *ctx, int64_t rows, int64_t cols, int64_t nnz,
                                               const int64_t *d_rowptr, const int32_t *d_colidx,
                                               const int32_t *d_vals, wr_matrix **out) {
    if (ctx && (ctx->chain_reduce || ctx->reorder)) {
        // the read-time passes run on the host: bring the CSR over first
        if (!out || !d_rowptr) return fail(WR_EINVAL, "null argument");
        if (rows < 0 || cols < 0 || nnz < 0) return fail(WR_EINVAL, "negative size");
        if (nnz > 0 && (!d_colidx || !d_vals)) return fail(WR_EINVAL, "null column or value array");
        WR_CUDA(cudaSetDevice(ctx->device));
        std::vector<int64_t> rp(rows + 1);
        std::vector<int32_t> ci(nnz), va(nnz);
        WR_CUDA(cudaMemcpyAsync(rp.data(), d_rowptr, sizeof(int64_t) * (rows + 1), cudaMemcpyDeviceToHost, ctx->stream));
        if (nnz > 0) {
            WR_CUDA(cudaMemcpyAsync(ci.data(), d_colidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, ctx->stream));
            WR_CUDA(cudaMemcpyAsync(va.data(), d_vals, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, ctx->stream));
        }
        WR_CUDA(cudaStreamSynchronize(ctx->stream));
        if (rp[rows] != nnz) return fail(WR_EINVAL, "rowptr[rows] must equal nnz");
        return load_prepared(ctx, rows, cols, rp.data(), ci.data(), va.data(), out);
    }
    WR_TRY(load_device(ctx, rows, cols, nnz, d_rowptr, d_colidx, d_vals, out));
    (*out)->rows_in = rows;
    (*out)->cols_in = cols;
    return WR_OK;
}

extern "C" wr_status wr_matrix_load_csr(wr_ctx *ctx, int64_t rows, int64_t cols, const int64_t *rowptr,
                                        const int32_t *colidx, const int32_t *vals, wr_matrix **out) {
    if (ctx && (ctx->chain_reduce || ctx->reorder)) return load_prepared(ctx, rows, cols, rowptr, colidx, vals, out);
    WR_TRY(load_host_plain(ctx, rows, cols, rowptr, colidx, vals, out));
    (*out)->rows_in = rows;
    (*out)->cols_in = cols;
    return WR_OK;
}

static wr_status load_host_plain(wr_ctx *ctx, int64_t rows, int64_t cols, const int64_t *rowptr,
                                 const int32_t *colidx, const int32_t *vals, wr_matrix **out) {
    if (!ctx || !out || !rowptr) return fail(WR_EINVAL, "null argument");
    if (rows < 0 || cols < 0) return fail(WR_EINVAL, "negative size");
    const int64_t nnz = rowptr[rows];
    if (nnz < 0) return fail(WR_EINVAL, "negative nnz");
    if (nnz > 0 && (!colidx || !vals)) return fail(WR_EINVAL, "null column or value array");
    WR_CUDA(cudaSetDevice(ctx->device));
    DevBuf rp, ci, va;
    WR_TRY(dev_alloc(ctx, rp, sizeof(int64_t) * (rows + 1)));
    WR_TRY(dev_alloc(ctx, ci, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    WR_TRY(dev_alloc(ctx, va, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    WR_CUDA(cudaMemcpyAsync(rp.ptr, rowptr, sizeof(int64_t) * (rows + 1), cudaMemcpyHostToDevice, ctx->stream));
    if (nnz > 0) {
        WR_CUDA(cudaMemcpyAsync(ci.ptr, colidx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, ctx->stream));
        WR_CUDA(cudaMemcpyAsync(va.ptr, vals, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, ctx->stream));
    }
    return load_device(ctx, rows, cols, nnz, rp.as<int64_t>(), ci.as<int32_t>(), va.as<int32_t>(), out);
}

extern "C" wr_status wr_set_locality_order(wr_ctx *ctx, int32_t on) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    ctx->reorder = on != 0;
    return WR_OK;
}

extern "C" wr_status wr_set_chain_reduction(wr_ctx *ctx, int32_t on) {
    if (!ctx) return fail(WR_EINVAL, "null context");
    ctx->chain_reduce = on != 0;
    return WR_OK;
}

extern "C" wr_status wr_matrix_reduction(const wr_matrix *mat, int64_t *rows_in, int64_t *cols_in,
                                         int64_t *rank_offset) {
    if (!mat) return fail(WR_EINVAL, "null matrix");
    if (rows_in) *rows_in = mat->rows_in;
    if (cols_in) *cols_in = mat->cols_in;
    if (rank_offset) *rank_offset = mat->rank_offset;
    return WR_OK;
}

extern "C" wr_status wr_matrix_info(const wr_matrix *mat, int64_t *rows, int64_t *cols, int64_t *nnz,
                                    int64_t *slots_a, int64_t *slots_at) {
    if (!mat) return fail(WR_EINVAL, "null matrix");
    if (rows) *rows = mat->rows;
    if (cols) *cols = mat->cols;
    if (nnz) *nnz = mat->nnz;
    if (slots_a) *slots_a = mat->a.nslots;
    if (slots_at) *slots_at = mat->at.nslots;
    return WR_OK;
}

extern "C" void wr_matrix_free(wr_matrix *mat) {
    if (!mat) return;
    cudaSetDevice(mat->ctx->device);
    cudaStreamSynchronize(mat->ctx->stream);
    delete mat;
}

// ------------------------------------------------------------------ rank

namespace wr {

void copy_settings(const wr_ctx *parent, wr_ctx *c) {
    c->profiling = parent->profiling;
    c->autotune = parent->autotune;
    c->lane_width = parent->lane_width;
    c->pair_generic = parent->pair_generic;
    c->pipeline = parent->pipeline;
    c->proj_overlap = parent->proj_overlap;
    c->early_term = parent->early_term;
    c->chain_reduce = parent->chain_reduce;
    c->reorder = parent->reorder;
    c->sigma_chunk = parent->sigma_chunk;
    c->sigma_leaf = parent->sigma_leaf;
    c->tensor_proj = parent->tensor_proj;
    c->slab_bytes = parent->slab_bytes;
    c->batch_fuse = parent->batch_fuse;
    c->alloc_fn = parent->alloc_fn;
    c->free_fn = parent->free_fn;
    c->alloc_user = parent->alloc_user;
}

// The greatest (high) or least stream priority of the device.
static int stream_priority(bool high) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    return high ? greatest : least;
}

wr_status make_child(const wr_ctx *parent, wr_ctx **out, bool high) {
    cudaStream_t s = nullptr;
    WR_CUDA(cudaSetDevice(parent->device));
    WR_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, stream_priority(high)));
    const wr_status st = wr_create(out, parent->device, s);
    if (st != WR_OK) {
        cudaStreamDestroy(s);
        return st;
    }
    (*out)->own_stream = true;
    (*out)->high_priority = high;
    copy_settings(parent, *out);
    return WR_OK;
}

// Which stream of a pipelined rank goes first: mode 2 the sigma-basis's, 3
// the sequence's, 1 (automatic) the sigma-basis's when it trails in PM-Basis
// segments (their kernels need most of an SM and wait long for SMs to drain
// of SpMM blocks, so without the priority they fall behind the terms) and
// the sequence's when the blocked M-Basis trails chunk by chunk (its kernels
// fill the gaps between the SpMM's).
static bool sigma_goes_first(const wr_ctx *ctx, int64_t L, int m, int n) {
    if (ctx->pipeline == 2) return true;
    if (ctx->pipeline == 3) return false;
    return sigma_pm_trailing(ctx, L, m, n);
}

// The pipeline's sequence stream at the greatest priority or at the least.
static wr_status ensure_seq_stream(wr_ctx *ctx, bool high) {
    if (ctx->seq_stream && ctx->seq_high == high) return WR_OK;
    if (ctx->seq_stream) {
        cudaStreamSynchronize(ctx->seq_stream);
        cudaStreamDestroy(ctx->seq_stream);
        ctx->seq_stream = nullptr;
    }
    cudaError_t ce = cudaStreamCreateWithPriority(&ctx->seq_stream, cudaStreamNonBlocking, stream_priority(high));
    if (ce != cudaSuccess) {
        ctx->seq_stream = nullptr;
        return cuda_fail(ce, "cudaStreamCreateWithPriority");
    }
    ctx->seq_high = high;
    return WR_OK;
}

wr_status feed_wait(wr_ctx *ctx, SeqFeed *feed, int64_t terms) {
    if (!feed || terms <= 0) return WR_OK;
    cudaEvent_t ev = nullptr;
    {
        std::unique_lock<std::mutex> lk(feed->mu);
        int64_t i = std::max<int64_t>(feed->waited, 0);
        for (;;) {
            while (i < (int64_t)feed->ready.size() && feed->ready[i] >= 0 && feed->ready[i] < terms) i++;
            if (i < (int64_t)feed->ready.size()) {
                if (feed->ready[i] < 0) return fail(WR_EDEVICE, "the sequence stopped before its terms were ready");
                break;
            }
            if (feed->closed) return fail(WR_EDEVICE, "the sequence stopped before its terms were ready");
            feed->cv.wait(lk);
        }
        if (i == feed->waited) return WR_OK;  // the stream already waits on that event
        feed->waited = i;
        ev = feed->ev[i];
    }
    WR_CUDA(cudaStreamWaitEvent(ctx->stream, ev, 0));
    return WR_OK;
}

// The readout of a finished sigma-basis into res (Section 2.5 step 4), the
// sequence copied back when wanted, and the Monte Carlo consistency checks.
static wr_status finish_result(wr_ctx *ctx, const wr_matrix *mat, const Resolved &r, const wr_params *params,
                               const DevBuf &dS, const DevBuf &dP, const DevBuf &ddeg, int64_t Dcap, int64_t L_used,
                               wr_result *res, double *readout_ms) {
    Readout ro;
    cudaEvent_t e1 = nullptr, e2 = nullptr;
    WR_CUDA(cudaEventCreate(&e1));
    WR_CUDA(cudaEventCreate(&e2));
    cudaEventRecord(e1, ctx->stream);
    wr_status st = rank_readout(ctx, dP.as<uint32_t>(), ddeg.as<int32_t>(), r.m, r.n, r.p, Dcap, ro,
                                (params->want & WR_WANT_GENERATOR) ? &res->gen : nullptr);
    if (st == WR_OK) {
        cudaEventRecord(e2, ctx->stream);
        cudaEventSynchronize(e2);
        float b = 0;
        cudaEventElapsedTime(&b, e1, e2);
        if (readout_ms) *readout_ms = b;
    }
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    WR_TRY(st);
    res->seq_len = L_used;
    if (params->want & WR_WANT_SEQUENCE) {
        res->seq.resize((size_t)L_used * r.m * r.n);
        cudaError_t e = cudaMemcpyAsync(res->seq.data(), dS.ptr, sizeof(uint32_t) * res->seq.size(),
                                        cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy sequence");
    }
    // Monte Carlo consistency: deg det F of a generator of X^T A~^i Y (A~ of
    // order N) is at most N, and 0 <= codeg <= deg det F
    if (ro.rank < 0 || ro.rank > r.N || ro.codeg < 0 || ro.deg_det > r.N)
        return fail(WR_EPROBFAIL, "inconsistent readout (rank " + std::to_string(ro.rank) + ", codeg " +
                                      std::to_string(ro.codeg) + ", deg det " + std::to_string(ro.deg_det) +
                                      "); retry with another seed");
    res->rank = mat->rank_offset + ro.rank;
    res->deg_det = ro.deg_det;
    res->codeg = ro.codeg;
    res->sum_delta = ro.sum_delta;
    if (params->want & WR_WANT_GENERATOR) {
        res->gen_deg = ro.delta;
        res->gen_dmax = ro.dmax;
    }
    return WR_OK;
}

wr_status rank_one(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params, wr_result **out) {
    if (!ctx || !mat || !params || !out) return fail(WR_EINVAL, "null argument");
    *out = nullptr;
    Resolved r;
    WR_TRY(resolve(mat, params, r));
    WR_CUDA(cudaSetDevice(ctx->device));
    ctx->last = wr_timings{};
    auto t_start = std::chrono::steady_clock::now();
    wr_result *res = new wr_result();
    res->prime = r.p;
    res->m = (uint32_t)r.m;
    res->n = (uint32_t)r.n;
    res->seq_len = r.L;
    if (r.N == 0) {
        res->rank = mat->rank_offset;
        *out = res;
        return WR_OK;
    }
    const int64_t L = r.L;
    const int q = r.m + r.n;
    const int64_t Dcap = L + 1;
    DevBuf dS, dP, ddeg;
    wr_status st = dev_alloc(ctx, dS, sizeof(uint32_t) * L * r.m * r.n);
    if (st == WR_OK) st = dev_alloc(ctx, dP, sizeof(uint32_t) * (Dcap + 1) * r.n * q);
    if (st == WR_OK) st = dev_alloc(ctx, ddeg, sizeof(int32_t) * q);
    double setup_ms = 0, seq_ms = 0, sigma_ms = 0, tail_ms = 0;
    int64_t L_used = L;  // terms the generator was computed from (< L after early termination)
    if (st == WR_OK && ctx->pipeline) {
        // The sigma-basis trails the sequence: a child context (own stream,
        // own host thread) runs M-Basis chunk k as soon as the sequence
        // stream has published S_0 .. S_{k+b-1}, so the two overlap on the
        // device and only the last chunks run after the sequence ends.
        // mode 1: the sequence's SpMM blocks go first wherever both phases
        // have blocks waiting and the sigma-basis fills the gaps; mode 2:
        // the sigma-basis first (its streams at the greatest priority)
        const bool sfirst = sigma_goes_first(ctx, L, r.m, r.n);
        if (ctx->aux && ctx->aux->high_priority != sfirst) {
            wr_destroy(ctx->aux);
            ctx->aux = nullptr;
        }
        if (!ctx->aux) st = make_child(ctx, &ctx->aux, sfirst);
        if (st == WR_OK) st = ensure_seq_stream(ctx, !sfirst);
        wr_ctx *aux = ctx->aux;
        SeqFeed feed;
        feed.throttle = ctx->early_term > 0 ? 3 : 0;
        cudaEvent_t ready0 = nullptr;
        if (st == WR_OK) {
            copy_settings(ctx, aux);
            aux->launches = 0;
            aux->last = wr_timings{};
            cudaError_t ce = cudaEventCreateWithFlags(&ready0, cudaEventDisableTiming);
            if (ce == cudaSuccess) ce = cudaEventRecord(ready0, ctx->stream);  // dS, dP, ddeg allocated
            if (ce != cudaSuccess) st = cuda_fail(ce, "cudaEventRecord");
        }
        if (st == WR_OK) {
            wr_status sst = WR_OK;
            std::string smsg;
            std::chrono::steady_clock::time_point t_sig0, t_sig1;
            aux->feed = &feed;
            std::thread sig([&] {
                cudaSetDevice(aux->device);
                t_sig0 = std::chrono::steady_clock::now();
                cudaError_t ce = cudaStreamWaitEvent(aux->stream, ready0, 0);
                sst = ce == cudaSuccess ? WR_OK : cuda_fail(ce, "cudaStreamWaitEvent");
                if (sst == WR_OK)
                    sst = sigma_basis(aux, dS.as<uint32_t>(), L, r.m, r.n, r.p, dP.as<uint32_t>(),
                                      ddeg.as<int32_t>(), Dcap);
                if (sst == WR_OK) {
                    ce = sync_stream_blocking(aux->stream);
                    if (ce != cudaSuccess) sst = cuda_fail(ce, "cudaStreamSynchronize");
                }
                t_sig1 = std::chrono::steady_clock::now();
                if (sst != WR_OK) smsg = wr_last_error();
            });
            // the sequence on the high-priority stream, after what the
            // caller's stream holds so far (the allocations above)
            cudaStream_t user = ctx->stream;
            cudaError_t ce = cudaStreamWaitEvent(ctx->seq_stream, ready0, 0);
            if (ce != cudaSuccess) {
                st = cuda_fail(ce, "cudaStreamWaitEvent");
            } else {
                ctx->stream = ctx->seq_stream;
                st = run_sequence(ctx, mat, *params, L, dS.as<uint32_t>(), &setup_ms, &seq_ms, &feed);
                ctx->stream = user;
                // run_sequence waited for its last event; order the caller's
                // stream after the sequence stream all the same
                cudaEvent_t done_ev = nullptr;
                if (cudaEventCreateWithFlags(&done_ev, cudaEventDisableTiming) == cudaSuccess) {
                    cudaEventRecord(done_ev, ctx->seq_stream);
                    cudaStreamWaitEvent(user, done_ev, 0);
                    cudaEventDestroy(done_ev);
                }
            }
            const auto t_seq1 = std::chrono::steady_clock::now();
            {
                std::lock_guard<std::mutex> lk(feed.mu);
                feed.closed = true;
            }
            feed.cv.notify_all();
            sig.join();
            aux->feed = nullptr;
            ctx->launches += aux->launches;
            ctx->last.sigma_window_ms = aux->last.sigma_window_ms;
            ctx->last.sigma_local_ms = aux->last.sigma_local_ms;
            ctx->last.sigma_apply_ms = aux->last.sigma_apply_ms;
            ctx->last.sigma_product_ms = aux->last.sigma_product_ms;
            sigma_ms = std::chrono::duration<double, std::milli>(t_sig1 - t_sig0).count();
            tail_ms = std::max(0.0, std::chrono::duration<double, std::milli>(t_sig1 - t_seq1).count());
            if (st == WR_OK && sst != WR_OK) st = fail(sst, smsg);
            if (feed.orders_used >= 0 && feed.orders_used < L) L_used = feed.orders_used;
        }
        for (cudaEvent_t e : feed.ev) cudaEventDestroy(e);
        if (ready0) cudaEventDestroy(ready0);
    } else if (st == WR_OK) {
        st = run_sequence(ctx, mat, *params, L, dS.as<uint32_t>(), &setup_ms, &seq_ms);
        const auto t0 = std::chrono::steady_clock::now();
        if (st == WR_OK)
            st = sigma_basis(ctx, dS.as<uint32_t>(), L, r.m, r.n, r.p, dP.as<uint32_t>(), ddeg.as<int32_t>(), Dcap);
        if (st == WR_OK) {
            cudaError_t ce = cudaStreamSynchronize(ctx->stream);
            if (ce != cudaSuccess) st = cuda_fail(ce, "cudaStreamSynchronize");
        }
        sigma_ms = tail_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    double readout_ms = 0;
    if (st == WR_OK) st = finish_result(ctx, mat, r, params, dS, dP, ddeg, Dcap, L_used, res, &readout_ms);
    if (st != WR_OK) {
        delete res;
        return st;
    }
    ctx->last.setup_ms = setup_ms;
    ctx->last.sequence_ms = seq_ms;
    ctx->last.sigma_ms = sigma_ms;
    ctx->last.sigma_tail_ms = tail_ms;
    ctx->last.readout_ms = readout_ms;
    ctx->last.total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    *out = res;
    return WR_OK;
}

// Several jobs on one matrix (same m = n, side and length; any primes and
// seeds, for the rank over Q by several primes, Section 2.5): one sequence
// loop for all of them (run_sequence_multi), then each job's sigma-basis on a
// stream of its own (concurrently), then each readout.  outs[g] receives job
// g's result, bit-identical to rank_one's.
wr_status rank_multi(wr_ctx *ctx, const wr_matrix *mat, const wr_params *const *params, int G, wr_result **outs) {
    if (!ctx || !mat || !params || !outs || G < 1 || G > MULTI_MAX_JOBS) return fail(WR_EINVAL, "bad multi-job call");
    for (int g = 0; g < G; g++) outs[g] = nullptr;
    WR_CUDA(cudaSetDevice(ctx->device));
    std::vector<Resolved> rs(G);
    for (int g = 0; g < G; g++) WR_TRY(resolve(mat, params[g], rs[g]));
    const Resolved &r0 = rs[0];
    if (r0.N == 0) {
        for (int g = 0; g < G; g++) WR_TRY(rank_one(ctx, mat, params[g], &outs[g]));
        return WR_OK;
    }
    const int64_t L = r0.L, Dcap = L + 1;
    const int q = r0.m + r0.n;
    std::vector<DevBuf> dS(G), dP(G), ddeg(G);
    std::vector<uint32_t *> pS(G);
    for (int g = 0; g < G; g++) {
        WR_TRY(dev_alloc(ctx, dS[g], sizeof(uint32_t) * L * r0.m * r0.n));
        WR_TRY(dev_alloc(ctx, dP[g], sizeof(uint32_t) * (Dcap + 1) * r0.n * q));
        WR_TRY(dev_alloc(ctx, ddeg[g], sizeof(int32_t) * q));
        pS[g] = dS[g].as<uint32_t>();
    }
    double seq_ms = 0;
    // The sigma-bases, each on a child context of its own; with the pipeline
    // they trail the shared sequence (each fed by its job's published terms)
    // while it runs on the high-priority sequence stream.
    std::vector<wr_ctx *> kids(G, nullptr);
    wr_status st = WR_OK;
    const bool piped = ctx->pipeline != 0;
    const bool sfirst = piped && sigma_goes_first(ctx, L, r0.m, r0.n);
    for (int g = 0; g < G && st == WR_OK; g++) {
        st = make_child(ctx, &kids[g], sfirst);
        if (st == WR_OK) copy_settings(ctx, kids[g]);
    }
    if (st == WR_OK && piped) st = ensure_seq_stream(ctx, !sfirst);
    std::vector<std::unique_ptr<SeqFeed>> feeds;
    std::vector<SeqFeed *> fptr;
    cudaEvent_t ready0 = nullptr;
    if (st == WR_OK && piped) {
        for (int g = 0; g < G; g++) {
            feeds.emplace_back(new SeqFeed());
            fptr.push_back(feeds.back().get());
            kids[g]->feed = fptr.back();
        }
        cudaError_t ce = cudaEventCreateWithFlags(&ready0, cudaEventDisableTiming);
        if (ce == cudaSuccess) ce = cudaEventRecord(ready0, ctx->stream);  // the buffers above are allocated
        if (ce != cudaSuccess) st = cuda_fail(ce, "cudaEventRecord");
    }
    if (st == WR_OK && !piped) st = run_sequence_multi(ctx, mat, rs, pS, &seq_ms);
    if (st == WR_OK) {
        std::vector<wr_status> sst(G, WR_OK);
        std::vector<std::string> smsg(G);
        std::vector<std::thread> th;
        for (int g = 0; g < G; g++)
            th.emplace_back([&, g] {
                cudaSetDevice(ctx->device);
                if (piped) {
                    cudaError_t ce = cudaStreamWaitEvent(kids[g]->stream, ready0, 0);
                    if (ce != cudaSuccess) { sst[g] = cuda_fail(ce, "cudaStreamWaitEvent"); smsg[g] = wr_last_error(); return; }
                }
                sst[g] = sigma_basis(kids[g], pS[g], L, r0.m, r0.n, rs[g].p, dP[g].as<uint32_t>(),
                                     ddeg[g].as<int32_t>(), Dcap);
                if (sst[g] == WR_OK) {
                    cudaError_t ce = sync_stream_blocking(kids[g]->stream);
                    if (ce != cudaSuccess) sst[g] = cuda_fail(ce, "cudaStreamSynchronize");
                }
                if (sst[g] != WR_OK) smsg[g] = wr_last_error();
            });
        if (piped) {
            cudaStream_t user = ctx->stream;
            cudaError_t ce = cudaStreamWaitEvent(ctx->seq_stream, ready0, 0);
            if (ce != cudaSuccess) {
                st = cuda_fail(ce, "cudaStreamWaitEvent");
            } else {
                ctx->stream = ctx->seq_stream;
                st = run_sequence_multi(ctx, mat, rs, pS, &seq_ms, &fptr);
                ctx->stream = user;
                cudaEvent_t done_ev = nullptr;
                if (cudaEventCreateWithFlags(&done_ev, cudaEventDisableTiming) == cudaSuccess) {
                    cudaEventRecord(done_ev, ctx->seq_stream);
                    cudaStreamWaitEvent(user, done_ev, 0);
                    cudaEventDestroy(done_ev);
                }
            }
            for (auto *fd : fptr) {
                {
                    std::lock_guard<std::mutex> lk(fd->mu);
                    fd->closed = true;
                }
                fd->cv.notify_all();
            }
        }
        for (auto &t : th) t.join();
        for (int g = 0; g < G && st == WR_OK; g++)
            if (sst[g] != WR_OK) st = fail(sst[g], smsg[g]);
    }
    for (auto *k : kids)
        if (k) {
            ctx->launches += k->launches;
            k->feed = nullptr;
            wr_destroy(k);
        }
    for (auto *fd : fptr)
        for (cudaEvent_t e : fd->ev) cudaEventDestroy(e);
    if (ready0) cudaEventDestroy(ready0);
    WR_TRY(st);
    for (int g = 0; g < G; g++) {
        wr_result *res = new wr_result();
        res->prime = rs[g].p;
        res->m = (uint32_t)r0.m;
        res->n = (uint32_t)r0.n;
        wr_status fs = finish_result(ctx, mat, rs[g], params[g], dS[g], dP[g], ddeg[g], Dcap, L, res, nullptr);
        if (fs != WR_OK) {
            delete res;
            for (int h = 0; h < g; h++) {
                delete outs[h];
                outs[h] = nullptr;
            }
            return fs;
        }
        outs[g] = res;
    }
    ctx->last.sequence_ms = seq_ms;
    return WR_OK;
}

}  // namespace wr

extern "C" wr_status wr_rank(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params, wr_result **out) {
    return rank_one(ctx, mat, params, out);
}

extern "C" uint64_t wr_result_rank(const wr_result *res) { return res ? (uint64_t)res->rank : 0; }

extern "C" wr_status wr_result_info(const wr_result *res, int64_t *deg_det, int64_t *codeg, int64_t *sum_delta,
                                    int64_t *seq_len) {
    if (!res) return fail(WR_EINVAL, "null result");
    if (deg_det) *deg_det = res->deg_det;
    if (codeg) *codeg = res->codeg;
    if (sum_delta) *sum_delta = res->sum_delta;
    if (seq_len) *seq_len = res->seq_len;
    return WR_OK;
}

extern "C" wr_status wr_result_sequence(const wr_result *res, uint32_t *dst, size_t cap_elems) {
    if (!res || !dst) return fail(WR_EINVAL, "null argument");
    if (res->seq.empty() && res->seq_len > 0 && res->m > 0)
        return fail(WR_EINVAL, "the sequence was not kept (WR_WANT_SEQUENCE)");
    if (cap_elems < res->seq.size()) return fail(WR_EINVAL, "destination too small");
    std::memcpy(dst, res->seq.data(), sizeof(uint32_t) * res->seq.size());
    return WR_OK;
}

extern "C" wr_status wr_result_generator(const wr_result *res, uint32_t *coeffs, size_t cap_elems,
                                         int32_t *col_degrees) {
    if (!res) return fail(WR_EINVAL, "null result");
    if (res->gen_dmax < 0) return fail(WR_EINVAL, "the generator was not kept (WR_WANT_GENERATOR)");
    if (coeffs) {
        if (cap_elems < res->gen.size()) return fail(WR_EINVAL, "destination too small");
        std::memcpy(coeffs, res->gen.data(), sizeof(uint32_t) * res->gen.size());
    }
    if (col_degrees) std::memcpy(col_degrees, res->gen_deg.data(), sizeof(int32_t) * res->gen_deg.size());
    return WR_OK;
}

extern "C" void wr_result_free(wr_result *res) { delete res; }

// ------------------------------------------------------------------ step-level calls

extern "C" wr_status wr_blackbox_apply_device(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                                              const uint32_t *d_in, uint32_t *d_out, int64_t width) {
    if (!ctx || !mat || !params || !d_in || !d_out) return fail(WR_EINVAL, "null argument");
    WR_CUDA(cudaSetDevice(ctx->device));
    return blackbox_apply(ctx, mat, *params, d_in, d_out, width);
}

// The paper has no counterpart: see the declaration in wr.h.
extern "C" wr_status wr_blackbox_apply_device_noalloc(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                                                      const uint32_t *d_in, uint32_t *d_out, int64_t width) {
    if (!ctx || !mat || !params || !d_in || !d_out) return fail(WR_EINVAL, "null argument");
    WR_CUDA(cudaSetDevice(ctx->device));
    return blackbox_apply_noalloc(ctx, mat, *params, d_in, d_out, width);
}

extern "C" wr_status wr_sequence_device(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                                        uint32_t *d_S, uint64_t L) {
    if (!ctx || !mat || !params || !d_S) return fail(WR_EINVAL, "null argument");
    Resolved r;
    WR_TRY(resolve(mat, params, r));
    WR_CUDA(cudaSetDevice(ctx->device));
    ctx->last = wr_timings{};
    if (r.N == 0) {
        WR_CUDA(cudaMemsetAsync(d_S, 0, sizeof(uint32_t) * L * r.m * r.n, ctx->stream));
        return WR_OK;
    }
    double a = 0, b = 0;
    WR_TRY(run_sequence(ctx, mat, *params, (int64_t)L, d_S, &a, &b));
    ctx->last.setup_ms = a;
    ctx->last.sequence_ms = b;
    return WR_OK;
}

extern "C" wr_status wr_sequence_state_device(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                                              uint32_t *d_S, uint64_t L, int64_t snap_at, uint32_t *d_snap,
                                              uint32_t *d_last, int64_t *applications, int32_t *paired) {
    if (!ctx || !mat || !params || !d_S) return fail(WR_EINVAL, "null argument");
    if (d_snap && snap_at < 0) return fail(WR_EINVAL, "snap_at must be >= 0 when d_snap is given");
    Resolved r;
    WR_TRY(resolve(mat, params, r));
    if (r.N == 0) return fail(WR_EINVAL, "the matrix has no rows or no columns");
    WR_CUDA(cudaSetDevice(ctx->device));
    ctx->last = wr_timings{};
    StateOut so;
    so.snap_at = d_snap ? snap_at : -1;
    so.d_snap = d_snap;
    so.d_last = d_last;
    double a = 0, b = 0;
    WR_TRY(run_sequence(ctx, mat, *params, (int64_t)L, d_S, &a, &b, nullptr, &so));
    if (d_snap && so.snap_at > so.applications)
        return fail(WR_EINVAL, "snap_at is beyond the applications of this sequence");
    ctx->last.setup_ms = a;
    ctx->last.sequence_ms = b;
    if (applications) *applications = so.applications;
    if (paired) *paired = so.paired ? 1 : 0;
    return WR_OK;
}

extern "C" wr_status wr_gram_device(wr_ctx *ctx, uint32_t prime, int64_t N, uint32_t m, uint32_t n,
                                    const uint32_t *d_t, int32_t tstride, int32_t yoff, const uint32_t *d_w,
                                    uint32_t *d_G) {
    if (!ctx || (N > 0 && (!d_t || !d_w)) || !d_G) return fail(WR_EINVAL, "null argument");
    if (prime <= 2 || prime >= (1u << 31) || !is_prime_u32(prime)) return fail(WR_ENOTPRIME, "bad prime");
    WR_CUDA(cudaSetDevice(ctx->device));
    return gram_device(ctx, prime, N, (int)m, (int)n, d_t, tstride, yoff, d_w, d_G);
}

extern "C" wr_status wr_polymat_mul_device(wr_ctx *ctx, uint32_t prime, const uint32_t *d_A, int64_t na,
                                           const uint32_t *d_B, int64_t nb, uint32_t r, uint32_t s, uint32_t t,
                                           int64_t lo, int64_t hi, uint32_t *d_C) {
    if (!ctx) return fail(WR_EINVAL, "null argument");
    if (na < 0 || nb < 0 || lo < 0 || lo > hi) return fail(WR_EINVAL, "na, nb >= 0 and 0 <= lo <= hi");
    if (r < 1 || s < 1 || t < 1 || r > 1024 || s > 1024 || t > 1024) return fail(WR_EINVAL, "r, s, t in 1..1024");
    if (prime <= 2 || prime >= (1u << 31) || !is_prime_u32(prime)) return fail(WR_ENOTPRIME, "bad prime");
    if (hi > lo && (!d_C || (na > 0 && nb > 0 && (!d_A || !d_B)))) return fail(WR_EINVAL, "null argument");
    WR_CUDA(cudaSetDevice(ctx->device));
    WR_TRY(polymat_mul(ctx, d_A, na, d_B, nb, (int)r, (int)s, (int)t, lo, hi, prime, d_C));
    WR_CUDA(cudaStreamSynchronize(ctx->stream));
    return WR_OK;
}

extern "C" wr_status wr_probe_mma(wr_ctx *ctx, int64_t iters, int32_t blocks, float *d_out, double *ms) {
    if (!ctx || !ms) return fail(WR_EINVAL, "null argument");
    if (iters < 1 || blocks < 1 || blocks > 4096) return fail(WR_EINVAL, "iters >= 1 and blocks in 1..4096");
    WR_CUDA(cudaSetDevice(ctx->device));
    return probe_mma(ctx, iters, blocks, d_out, ms);
}

extern "C" wr_status wr_sequence_slab_device(wr_ctx *ctx, const wr_matrix *mat, const wr_params *params,
                                             uint32_t col0, uint32_t ncols, uint32_t *d_S, uint64_t L) {
    if (!ctx || !mat || !params || !d_S) return fail(WR_EINVAL, "null argument");
    Resolved r;
    WR_TRY(resolve(mat, params, r));
    if (ncols < 1 || (uint64_t)col0 + ncols > (uint64_t)params->n)
        return fail(WR_EINVAL, "column slab [col0, col0 + ncols) must lie in [0, n) and be nonempty");
    WR_CUDA(cudaSetDevice(ctx->device));
    ctx->last = wr_timings{};
    r.n = (int)ncols;
    r.nv = padded_width(r.n);
    r.nvs = r.nv;
    r.ycol0 = (int)col0;
    r.gram = false;  // one term per application: X spans the whole Y, the right block is a slab
    if (r.N == 0) {
        WR_CUDA(cudaMemsetAsync(d_S, 0, sizeof(uint32_t) * L * r.m * r.n, ctx->stream));
        return WR_OK;
    }
    double a = 0, b = 0;
    WR_TRY(run_sequence_resolved(ctx, mat, r, (int64_t)L, d_S, &a, &b));
    ctx->last.setup_ms = a;
    ctx->last.sequence_ms = b;
    return WR_OK;
}

extern "C" wr_status wr_sigma_basis_device(wr_ctx *ctx, const uint32_t *d_S, uint64_t L, uint32_t m, uint32_t n,
                                           uint32_t prime, uint32_t *d_P, int32_t *d_deg, int64_t Dcap) {
    if (!ctx || !d_S || !d_P || !d_deg) return fail(WR_EINVAL, "null argument");
    if (prime <= 2 || prime >= (1u << 31) || !is_prime_u32(prime)) return fail(WR_ENOTPRIME, "bad prime");
    if (Dcap < (int64_t)L + 1) return fail(WR_EINVAL, "Dcap must be at least L + 1");
    WR_CUDA(cudaSetDevice(ctx->device));
    return sigma_basis(ctx, d_S, (int64_t)L, (int)m, (int)n, prime, d_P, d_deg, Dcap);
}

extern "C" wr_status wr_det_valuation_device(wr_ctx *ctx, const uint32_t *d_G, int64_t n, int64_t T, uint32_t prime,
                                             int64_t *val) {
    if (!ctx || !d_G || !val) return fail(WR_EINVAL, "null argument");
    if (prime <= 2 || prime >= (1u << 31) || !is_prime_u32(prime)) return fail(WR_ENOTPRIME, "bad prime");
    WR_CUDA(cudaSetDevice(ctx->device));
    return det_valuation(ctx, d_G, n, T, prime, val);
}
