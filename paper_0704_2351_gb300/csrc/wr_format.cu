// Matrix ingest on the device: CSR validation, exclusive scans, CSR
// transpose, and the SELL-C-sigma layout the SpMM kernels read.
//
// The paper reads its boundary matrices once and keeps them for the whole
// sequence (Section 2.6.4 reduces them at read time; Section 3.1 broadcasts
// A to every process).  Here the matrix is laid out once per load, in device
// memory, for both A and A^T (the two sparse passes of A~ = D1 A^T D2 A D1).
#include <cuda_runtime.h>

#include <algorithm>

#include "wr_internal.cuh"

namespace wr {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

enum : int { ERR_ROWPTR = 1, ERR_COL = 2, ERR_VAL = 4, ERR_ROWLEN = 8, ERR_WIDEVAL = 16, ERR_ROWLEN16 = 32 };

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t &excl) {
    __shared__ int64_t warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x / 32) ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int64_t warp_prefix = warp > 0 ? warp_sums[warp - 1] : 0;
    int64_t total = warp_sums[blockDim.x / 32 - 1];
    excl = warp_prefix + x - v;
    __syncthreads();
    return total;
}

__global__ void k_tile_sums(const int64_t *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) s += in[i];
    }
    int64_t excl;
    int64_t tot = block_exclusive_scan(s, excl);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_tile_scan(const int64_t *__restrict__ in, int64_t n, const int64_t *__restrict__ offs,
                            int64_t *__restrict__ out) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t loc[SCAN_ITEMS];
    int64_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        loc[k] = i < n ? in[i] : 0;
        s += loc[k];
    }
    int64_t excl;
    int64_t tot = block_exclusive_scan(s, excl);
    int64_t run = excl + (offs ? offs[blockIdx.x] : 0);
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) out[i] = run;
        run += loc[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
        (void)tot;
        out[n] = run;  // total
    }
}

// --- validation

__global__ void k_validate(int64_t rows, int64_t cols, int64_t nnz, const int64_t *__restrict__ rowptr,
                           const int32_t *__restrict__ colidx, const int32_t *__restrict__ vals,
                           int *__restrict__ err) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int e = 0;
    for (int64_t i = tid; i < rows; i += stride) {
        int64_t a = rowptr[i], b = rowptr[i + 1];
        if (b < a || a < 0 || b > nnz) e |= ERR_ROWPTR;
        else if (b - a >= (int64_t(1) << 24)) e |= ERR_ROWLEN;
        else if (b - a >= (int64_t(1) << 16)) e |= ERR_ROWLEN16;
    }
    if (tid == 0 && (rowptr[0] != 0 || rowptr[rows] != nnz)) e |= ERR_ROWPTR;
    for (int64_t k = tid; k < nnz; k += stride) {
        int32_t c = colidx[k];
        int32_t v = vals[k];
        if (c < 0 || c >= cols) e |= ERR_COL;
        if (v < -32767 || v > 32767) e |= ERR_VAL;
        else if (v < -127 || v > 127) e |= ERR_WIDEVAL;
    }
    if (e) atomicOr(err, e);
}

// --- transpose

__global__ void k_count_cols(int64_t nnz, const int32_t *__restrict__ colidx, int64_t *__restrict__ cnt) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = tid; k < nnz; k += stride)
        atomicAdd((unsigned long long *)&cnt[colidx[k]], 1ull);
}

__global__ void k_scatter_transpose(int64_t rows, const int64_t *__restrict__ rowptr,
                                    const int32_t *__restrict__ colidx, const int32_t *__restrict__ vals,
                                    const int64_t *__restrict__ rowptr_t, int64_t *__restrict__ fill,
                                    int32_t *__restrict__ colidx_t, int32_t *__restrict__ vals_t) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < rows; i += stride) {
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
            int32_t c = colidx[k];
            int64_t pos = rowptr_t[c] + (int64_t)atomicAdd((unsigned long long *)&fill[c], 1ull);
            colidx_t[pos] = (int32_t)i;
            vals_t[pos] = vals[k];
        }
    }
}

// --- layout build
//
// Light rows (at most LIGHT_MAX entries, empty rows included) go to the SELL
// part: sorted by length (descending), 32 per chunk, slot-major.  Longer rows
// go to the vector part: their entries are copied contiguously and cut into
// segments of at most VSEG entries; a row with more than one segment is a
// split row (exact int64 partial sums, finished by a second kernel).

__global__ void k_classify(int64_t rows, const int64_t *__restrict__ rowptr, int64_t *__restrict__ nseg,
                           int64_t *__restrict__ vlen, int64_t *__restrict__ is_split, int *__restrict__ hist,
                           int *__restrict__ err) {
    __shared__ int sh[LIGHT_MAX + 1];
    for (int b = threadIdx.x; b <= LIGHT_MAX; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < rows; i += stride) {
        const int64_t len = rowptr[i + 1] - rowptr[i];
        if (len >= (int64_t(1) << 24)) atomicOr(err, ERR_ROWLEN);
        if (len <= LIGHT_MAX) {
            nseg[i] = 0;
            vlen[i] = 0;
            is_split[i] = 0;
            atomicAdd(&sh[len], 1);
        } else {
            const int64_t ns = (len + VSEG - 1) / VSEG;
            nseg[i] = ns;
            vlen[i] = len;
            is_split[i] = ns > 1 ? 1 : 0;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b <= LIGHT_MAX; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

// bucket b (rows of length b) starts after all longer buckets
__global__ void k_bucket_starts(const int *__restrict__ hist, int64_t *__restrict__ start) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t run = 0;
        for (int b = LIGHT_MAX; b >= 0; b--) {
            start[b] = run;
            run += hist[b];
        }
        start[LIGHT_MAX + 1] = run;  // number of light rows
    }
}

__global__ void k_bucket_scatter(int64_t rows, const int64_t *__restrict__ rowptr,
                                 const int64_t *__restrict__ start, unsigned long long *__restrict__ fill,
                                 int32_t *__restrict__ sorted) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < rows; i += stride) {
        const int64_t len = rowptr[i + 1] - rowptr[i];
        if (len > LIGHT_MAX) continue;
        const int64_t pos = start[len] + (int64_t)atomicAdd(&fill[len], 1ull);
        sorted[pos] = (int32_t)i;
    }
}

__global__ void k_chunk_slots(int64_t nchunks, const int32_t *__restrict__ sorted,
                              const int64_t *__restrict__ rowptr, int32_t *__restrict__ chunk_len,
                              int64_t *__restrict__ slots) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = tid; c < nchunks; c += stride) {
        // sorted by length descending: the chunk's first row is its longest
        const int32_t r = sorted[c * SELL_C];
        const int l = (int)(rowptr[r + 1] - rowptr[r]);
        chunk_len[c] = l;
        slots[c] = (int64_t)l * SELL_C;
    }
}

__global__ void k_fill_light(int64_t nchunks, int64_t nlight, const int32_t *__restrict__ sorted,
                             const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                             const int32_t *__restrict__ vals, const int64_t *__restrict__ chunk_off,
                             const int32_t *__restrict__ chunk_len, uint32_t *__restrict__ entries,
                             uint32_t *__restrict__ vrow, int16_t *__restrict__ wvals) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t pos = tid; pos < nchunks * SELL_C; pos += stride) {
        const int64_t c = pos / SELL_C;
        const int lane = (int)(pos % SELL_C);
        const int clen = chunk_len[c];
        uint32_t *dst = entries + chunk_off[c] + lane;
        if (pos < nlight) {
            const int32_t r = sorted[pos];
            const int64_t s = rowptr[r];
            const int l = (int)(rowptr[r + 1] - s);
            int16_t *wdst = wvals ? wvals + chunk_off[c] + lane : nullptr;
            for (int j = 0; j < clen; j++) {
                uint32_t w = 0;
                if (wdst) {  // wide: the column in the entry word, the value beside it
                    if (j < l) w = (uint32_t)colidx[s + j];
                    wdst[(int64_t)j * SELL_C] = j < l ? (int16_t)vals[s + j] : (int16_t)0;
                } else if (j < l) {
                    w = ((uint32_t)colidx[s + j] << 8) | ((uint32_t)vals[s + j] & 0xFFu);
                }
                dst[(int64_t)j * SELL_C] = w;
            }
            vrow[pos] = (uint32_t)r;
        } else {
            for (int j = 0; j < clen; j++) dst[(int64_t)j * SELL_C] = 0;
            if (wvals)
                for (int j = 0; j < clen; j++) wvals[chunk_off[c] + lane + (int64_t)j * SELL_C] = 0;
            vrow[pos] = VROW_EMPTY;
        }
    }
}

// one warp per long row: copy its entries contiguously and write its segments
__global__ void k_fill_vector(int64_t rows, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                              const int32_t *__restrict__ vals, const int64_t *__restrict__ vlen,
                              const int64_t *__restrict__ voff, const int64_t *__restrict__ segbase,
                              const int64_t *__restrict__ is_split, const int64_t *__restrict__ split_id,
                              uint32_t *__restrict__ ventries, int64_t *__restrict__ seg_start,
                              int32_t *__restrict__ seg_len, uint32_t *__restrict__ seg_row,
                              int32_t *__restrict__ split_row, int16_t *__restrict__ vwvals) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < rows; i += nwarps) {
        const int64_t len = vlen[i];
        if (len == 0) continue;
        const int64_t s = rowptr[i], o = voff[i];
        if (vwvals) {
            for (int64_t j = lane; j < len; j += 32) {
                ventries[o + j] = (uint32_t)colidx[s + j];
                vwvals[o + j] = (int16_t)vals[s + j];
            }
        } else {
            for (int64_t j = lane; j < len; j += 32)
                ventries[o + j] = ((uint32_t)colidx[s + j] << 8) | ((uint32_t)vals[s + j] & 0xFFu);
        }
        const int64_t ns = (len + VSEG - 1) / VSEG;
        const uint32_t tgt = is_split[i] ? (VROW_SPLIT | (uint32_t)split_id[i]) : (uint32_t)i;
        for (int64_t k = lane; k < ns; k += 32) {
            const int64_t g = segbase[i] + k;
            seg_start[g] = o + k * VSEG;
            seg_len[g] = (int32_t)min64(VSEG, len - k * VSEG);
            seg_row[g] = tgt;
        }
        if (lane == 0 && is_split[i]) split_row[split_id[i]] = (int32_t)i;
    }
}

int grid_for(wr_ctx *ctx, int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)ctx->num_sms * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

wr_status read_err(wr_ctx *ctx, int *d_err, int *h_err) {
    WR_CUDA(cudaMemcpyAsync(h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    WR_CUDA(cudaStreamSynchronize(ctx->stream));
    return WR_OK;
}

}  // namespace

wr_status exclusive_scan_i64(wr_ctx *ctx, const int64_t *d_in, int64_t *d_out, int64_t n) {
    if (n <= 0) {
        WR_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int64_t), ctx->stream));
        return WR_OK;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_tile_scan<<<1, SCAN_THREADS, 0, ctx->stream>>>(d_in, n, nullptr, d_out);
        WR_LAUNCHED(ctx);
        return WR_OK;
    }
    DevBuf sums, offs;
    WR_TRY(dev_alloc(ctx, sums, sizeof(int64_t) * tiles));
    WR_TRY(dev_alloc(ctx, offs, sizeof(int64_t) * (tiles + 1)));
    k_tile_sums<<<(unsigned)tiles, SCAN_THREADS, 0, ctx->stream>>>(d_in, n, sums.as<int64_t>());
    WR_LAUNCHED(ctx);
    WR_TRY(exclusive_scan_i64(ctx, sums.as<int64_t>(), offs.as<int64_t>(), tiles));
    k_tile_scan<<<(unsigned)tiles, SCAN_THREADS, 0, ctx->stream>>>(d_in, n, offs.as<int64_t>(), d_out);
    WR_LAUNCHED(ctx);
    // the last tile wrote out[n]; keep the stream ordered for the caller
    return WR_OK;
}

// Checks a CSR matrix; *wide (in: already wide because of the dimensions;
// out: wide) selects the layout with 32-bit columns and int16 values, needed
// for entries outside [-127, 127] or dimensions of 2^24 and more.
wr_status validate_csr(wr_ctx *ctx, int64_t rows, int64_t cols, int64_t nnz, const int64_t *d_rowptr,
                       const int32_t *d_colidx, const int32_t *d_vals, bool *wide) {
    DevBuf err;
    WR_TRY(dev_alloc(ctx, err, sizeof(int)));
    WR_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), ctx->stream));
    int threads = 256;
    k_validate<<<grid_for(ctx, std::max(rows, nnz), threads), threads, 0, ctx->stream>>>(
        rows, cols, nnz, d_rowptr, d_colidx, d_vals, err.as<int>());
    WR_LAUNCHED(ctx);
    int h = 0;
    WR_TRY(read_err(ctx, err.as<int>(), &h));
    if (h & ERR_ROWPTR) return fail(WR_EINVAL, "rowptr is not a valid CSR row pointer array");
    if (h & ERR_COL) return fail(WR_EINVAL, "column index out of range");
    if (h & ERR_VAL) return fail(WR_EOVERFLOW, "matrix entry outside [-32767, 32767]");
    if (h & ERR_ROWLEN) return fail(WR_EOVERFLOW, "a row holds 2^24 or more entries");
    if (h & ERR_WIDEVAL) *wide = true;
    if (*wide && (h & ERR_ROWLEN16))
        return fail(WR_EOVERFLOW, "with entries outside [-127, 127] (or a dimension of 2^24 or more) every row and "
                                  "column must hold fewer than 65,536 entries");
    return WR_OK;
}

wr_status transpose_csr(wr_ctx *ctx, int64_t rows, int64_t cols, int64_t nnz, const int64_t *d_rowptr,
                        const int32_t *d_colidx, const int32_t *d_vals, DevBuf &rowptr_t,
                        DevBuf &colidx_t, DevBuf &vals_t) {
    DevBuf cnt, fill;
    WR_TRY(dev_alloc(ctx, cnt, sizeof(int64_t) * (cols + 1)));
    WR_TRY(dev_alloc(ctx, fill, sizeof(int64_t) * (cols + 1)));
    WR_TRY(dev_alloc(ctx, rowptr_t, sizeof(int64_t) * (cols + 1)));
    WR_TRY(dev_alloc(ctx, colidx_t, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    WR_TRY(dev_alloc(ctx, vals_t, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    WR_CUDA(cudaMemsetAsync(cnt.ptr, 0, sizeof(int64_t) * (cols + 1), ctx->stream));
    WR_CUDA(cudaMemsetAsync(fill.ptr, 0, sizeof(int64_t) * (cols + 1), ctx->stream));
    int threads = 256;
    if (nnz > 0) {
        k_count_cols<<<grid_for(ctx, nnz, threads), threads, 0, ctx->stream>>>(nnz, d_colidx,
                                                                               cnt.as<int64_t>());
        WR_LAUNCHED(ctx);
    }
    WR_TRY(exclusive_scan_i64(ctx, cnt.as<int64_t>(), rowptr_t.as<int64_t>(), cols));
    if (nnz > 0) {
        k_scatter_transpose<<<grid_for(ctx, rows, threads), threads, 0, ctx->stream>>>(
            rows, d_rowptr, d_colidx, d_vals, rowptr_t.as<int64_t>(), fill.as<int64_t>(),
            colidx_t.as<int32_t>(), vals_t.as<int32_t>());
        WR_LAUNCHED(ctx);
    }
    return WR_OK;
}

// entries of each row whose column lies in [c0, c1)
__global__ void k_slab_count(int64_t rows, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                             int32_t c0, int32_t c1, int64_t *__restrict__ cnt) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int64_t k = 0;
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; e++) {
        const int32_t c = colidx[e];
        k += (c >= c0 && c < c1) ? 1 : 0;
    }
    cnt[r] = k;
}

__global__ void k_slab_fill(int64_t rows, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                            const int32_t *__restrict__ vals, int32_t c0, int32_t c1,
                            const int64_t *__restrict__ rowptr_s, int32_t *__restrict__ colidx_s,
                            int32_t *__restrict__ vals_s) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int64_t w = rowptr_s[r];
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; e++) {
        const int32_t c = colidx[e];
        if (c >= c0 && c < c1) {
            colidx_s[w] = c;
            vals_s[w] = vals[e];
            w++;
        }
    }
}

// The layout of the entries of a CSR whose columns lie in [c0, c1) (columns
// keep their numbers; every row of the matrix has a row in the layout, empty
// ones included, so that a pass over this slab writes every output row).
wr_status build_sell_slab(wr_ctx *ctx, int64_t rows, int64_t cols, const int64_t *d_rowptr, const int32_t *d_colidx,
                          const int32_t *d_vals, int32_t c0, int32_t c1, Sell &out, bool wide) {
    cudaStream_t st = ctx->stream;
    DevBuf cnt, rp;
    WR_TRY(dev_alloc(ctx, cnt, sizeof(int64_t) * (rows + 1)));
    WR_TRY(dev_alloc(ctx, rp, sizeof(int64_t) * (rows + 1)));
    if (rows > 0) {
        k_slab_count<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(rows, d_rowptr, d_colidx, c0, c1,
                                                                      cnt.as<int64_t>());
        WR_LAUNCHED(ctx);
    }
    WR_TRY(exclusive_scan_i64(ctx, cnt.as<int64_t>(), rp.as<int64_t>(), rows));
    int64_t nnz = 0;
    WR_CUDA(cudaMemcpyAsync(&nnz, rp.as<int64_t>() + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    WR_CUDA(cudaStreamSynchronize(st));
    DevBuf ci, va;
    WR_TRY(dev_alloc(ctx, ci, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    WR_TRY(dev_alloc(ctx, va, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    if (rows > 0) {
        k_slab_fill<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(rows, d_rowptr, d_colidx, d_vals, c0, c1,
                                                                     rp.as<int64_t>(), ci.as<int32_t>(),
                                                                     va.as<int32_t>());
        WR_LAUNCHED(ctx);
    }
    return build_sell(ctx, rows, cols, nnz, rp.as<int64_t>(), ci.as<int32_t>(), va.as<int32_t>(), out, wide);
}

wr_status build_sell(wr_ctx *ctx, int64_t rows, int64_t cols, int64_t nnz, const int64_t *d_rowptr,
                     const int32_t *d_colidx, const int32_t *d_vals, Sell &out, bool wide) {
    (void)nnz;
    out.nrows = rows;
    out.ncols = cols;
    out.wide = wide;
    const int threads = 256;
    cudaStream_t st = ctx->stream;
    const int64_t R1 = rows + 1;
    DevBuf nseg, vlen, is_split, segbase, voff, split_id, hist, bstart, bfill, err;
    WR_TRY(dev_alloc(ctx, nseg, sizeof(int64_t) * R1));
    WR_TRY(dev_alloc(ctx, vlen, sizeof(int64_t) * R1));
    WR_TRY(dev_alloc(ctx, is_split, sizeof(int64_t) * R1));
    WR_TRY(dev_alloc(ctx, segbase, sizeof(int64_t) * R1));
    WR_TRY(dev_alloc(ctx, voff, sizeof(int64_t) * R1));
    WR_TRY(dev_alloc(ctx, split_id, sizeof(int64_t) * R1));
    WR_TRY(dev_alloc(ctx, hist, sizeof(int) * (LIGHT_MAX + 1)));
    WR_TRY(dev_alloc(ctx, bstart, sizeof(int64_t) * (LIGHT_MAX + 2)));
    WR_TRY(dev_alloc(ctx, bfill, sizeof(unsigned long long) * (LIGHT_MAX + 1)));
    WR_TRY(dev_alloc(ctx, err, sizeof(int)));
    WR_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), st));
    WR_CUDA(cudaMemsetAsync(hist.ptr, 0, hist.bytes, st));
    WR_CUDA(cudaMemsetAsync(bfill.ptr, 0, bfill.bytes, st));
    if (rows > 0) {
        k_classify<<<grid_for(ctx, rows, threads), threads, 0, st>>>(rows, d_rowptr, nseg.as<int64_t>(),
                                                                    vlen.as<int64_t>(), is_split.as<int64_t>(),
                                                                    hist.as<int>(), err.as<int>());
        WR_LAUNCHED(ctx);
    }
    WR_TRY(exclusive_scan_i64(ctx, nseg.as<int64_t>(), segbase.as<int64_t>(), rows));
    WR_TRY(exclusive_scan_i64(ctx, vlen.as<int64_t>(), voff.as<int64_t>(), rows));
    WR_TRY(exclusive_scan_i64(ctx, is_split.as<int64_t>(), split_id.as<int64_t>(), rows));
    k_bucket_starts<<<1, 32, 0, st>>>(hist.as<int>(), bstart.as<int64_t>());
    WR_LAUNCHED(ctx);
    int64_t tot[4] = {0, 0, 0, 0};
    int herr = 0;
    WR_CUDA(cudaMemcpyAsync(&tot[0], segbase.as<int64_t>() + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    WR_CUDA(cudaMemcpyAsync(&tot[1], voff.as<int64_t>() + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    WR_CUDA(cudaMemcpyAsync(&tot[2], split_id.as<int64_t>() + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    WR_CUDA(cudaMemcpyAsync(&tot[3], bstart.as<int64_t>() + LIGHT_MAX + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    WR_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    WR_CUDA(cudaStreamSynchronize(st));
    if (herr & ERR_ROWLEN) return fail(WR_EOVERFLOW, "a row or column holds 2^24 or more entries");
    out.nseg = tot[0];
    out.nvent = tot[1];
    out.nsplit = tot[2];
    out.nlight = tot[3];
    out.nchunks = (out.nlight + SELL_C - 1) / SELL_C;

    // vector part
    WR_TRY(dev_alloc(ctx, out.ventries, sizeof(uint32_t) * std::max<int64_t>(out.nvent, 1)));
    WR_TRY(dev_alloc(ctx, out.seg_start, sizeof(int64_t) * std::max<int64_t>(out.nseg, 1)));
    WR_TRY(dev_alloc(ctx, out.seg_len, sizeof(int32_t) * std::max<int64_t>(out.nseg, 1)));
    WR_TRY(dev_alloc(ctx, out.seg_row, sizeof(uint32_t) * std::max<int64_t>(out.nseg, 1)));
    WR_TRY(dev_alloc(ctx, out.split_row, sizeof(int32_t) * std::max<int64_t>(out.nsplit, 1)));
    if (wide) WR_TRY(dev_alloc(ctx, out.vwvals, sizeof(int16_t) * std::max<int64_t>(out.nvent, 1)));
    if (out.nseg > 0) {
        k_fill_vector<<<grid_for(ctx, rows * 32, threads), threads, 0, st>>>(
            rows, d_rowptr, d_colidx, d_vals, vlen.as<int64_t>(), voff.as<int64_t>(), segbase.as<int64_t>(),
            is_split.as<int64_t>(), split_id.as<int64_t>(), out.ventries.as<uint32_t>(), out.seg_start.as<int64_t>(),
            out.seg_len.as<int32_t>(), out.seg_row.as<uint32_t>(), out.split_row.as<int32_t>(),
            wide ? out.vwvals.as<int16_t>() : nullptr);
        WR_LAUNCHED(ctx);
    }

    // light part
    DevBuf sorted, slots;
    WR_TRY(dev_alloc(ctx, sorted, sizeof(int32_t) * std::max<int64_t>(out.nchunks * SELL_C, 1)));
    WR_TRY(dev_alloc(ctx, slots, sizeof(int64_t) * (out.nchunks + 1)));
    WR_TRY(dev_alloc(ctx, out.chunk_off, sizeof(int64_t) * (out.nchunks + 1)));
    WR_TRY(dev_alloc(ctx, out.chunk_len, sizeof(int32_t) * std::max<int64_t>(out.nchunks, 1)));
    WR_TRY(dev_alloc(ctx, out.vrow, sizeof(uint32_t) * std::max<int64_t>(out.nchunks * SELL_C, 1)));
    if (out.nchunks == 0) {
        WR_CUDA(cudaMemsetAsync(out.chunk_off.ptr, 0, sizeof(int64_t), st));
        WR_TRY(dev_alloc(ctx, out.entries, sizeof(uint32_t)));
        if (wide) WR_TRY(dev_alloc(ctx, out.wvals, sizeof(int16_t)));
        out.nslots = 0;
        WR_CUDA(cudaStreamSynchronize(st));
        return WR_OK;
    }
    k_bucket_scatter<<<grid_for(ctx, rows, threads), threads, 0, st>>>(
        rows, d_rowptr, bstart.as<int64_t>(), bfill.as<unsigned long long>(), sorted.as<int32_t>());
    WR_LAUNCHED(ctx);
    k_chunk_slots<<<grid_for(ctx, out.nchunks, threads), threads, 0, st>>>(
        out.nchunks, sorted.as<int32_t>(), d_rowptr, out.chunk_len.as<int32_t>(), slots.as<int64_t>());
    WR_LAUNCHED(ctx);
    WR_TRY(exclusive_scan_i64(ctx, slots.as<int64_t>(), out.chunk_off.as<int64_t>(), out.nchunks));
    int64_t nslots = 0;
    WR_CUDA(cudaMemcpyAsync(&nslots, out.chunk_off.as<int64_t>() + out.nchunks, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, st));
    WR_CUDA(cudaStreamSynchronize(st));
    out.nslots = nslots;
    WR_TRY(dev_alloc(ctx, out.entries, sizeof(uint32_t) * std::max<int64_t>(nslots, 1)));
    if (wide) WR_TRY(dev_alloc(ctx, out.wvals, sizeof(int16_t) * std::max<int64_t>(nslots, 1)));
    k_fill_light<<<grid_for(ctx, out.nchunks * SELL_C, threads), threads, 0, st>>>(
        out.nchunks, out.nlight, sorted.as<int32_t>(), d_rowptr, d_colidx, d_vals, out.chunk_off.as<int64_t>(),
        out.chunk_len.as<int32_t>(), out.entries.as<uint32_t>(), out.vrow.as<uint32_t>(),
        wide ? out.wvals.as<int16_t>() : nullptr);
    WR_LAUNCHED(ctx);
    WR_CUDA(cudaStreamSynchronize(st));
    return WR_OK;
}

}  // namespace wr
