// The block Wiedemann sequence on the device (Section 2.5 step 2 of the paper;
// Section 2.2 for the block sequence X^T A~^i Y; Section 2.3 for A~).
//
// With T_k = D1 A~^k Y (stored, N x nv residues) the recurrence is
//   W       = D2 (A T_k)                    SpMM pass 1 (rows of A, or of A^T)
//   T_{k+1} = D1^2 (A^T W)                  SpMM pass 2 (the other layout)
//   S_{k+1} = Xh^T T_{k+1},  Xh = D1^{-1} X (so that S_k = X^T A~^k Y)
// Every row sum of a pass is exact in int64 (|a| <= 127, residues < 2^31,
// < 2^24 terms) and reduced once; the diagonal scaling is the epilogue.
// The paper's one-process-per-column scheme (Section 3.1) becomes the block
// width: all n columns of T ride on one pass over the matrix, each gathered
// row of T being one vector load of n residues.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "wr_internal.cuh"

#include "wr_spmm_kernel.cuh"

namespace wr {

namespace {

// S_raw[k] += Xh^T T (m x n), k = tmul * (term counter) + toff, skipped
// unless 0 <= k < L.  m threads per row (one per row of the block Xh^T), NV
// register accumulators each; rows are streamed over the grid.  Partials are
// reduced mod p before the exact uint64 atomics, so their sum cannot overflow
// and does not depend on the order.
// GRAM: the weighted Gram matrix sum_r wt[r] T[r]^T T[r] (m = n) instead; the
// symmetric projection X = Y turns every term into one (Section 2.3).  Rows
// of t are tstride residues apart; GRAM takes its left factor from the first
// m of them and the right one from yoff on (yoff > 0: the cross products of
// the paired block [D1 X | D1 Y]).
constexpr int PROJ_THREADS = 256;

template <int NV, int FOLDK, bool GRAM>
__global__ void __launch_bounds__(PROJ_THREADS)
    k_project(int64_t N, int m, int n, const uint32_t *__restrict__ xh, const uint32_t *__restrict__ t,
              unsigned long long *__restrict__ s_raw, const int *__restrict__ term_counter, int tmul, int toff,
              int64_t L, int tstride, int yoff, ModP mp) {
    const int64_t k_term = (int64_t)tmul * *term_counter + toff;
    if (k_term < 0 || k_term >= L) return;  // the same for every thread
    // red32[w][a][b]: per-warp sums reduced mod p (m divides 32); red: one
    // shared row of atomically added sums (other m)
    __shared__ uint32_t red32[(PROJ_THREADS / 32) * 32 * NV];
    __shared__ unsigned long long red[32 * NV];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool pow2 = (32 % m) == 0;
    const int per = PROJ_THREADS / m;  // rows per block step
    const int a = tid % m, slot = tid / m;
    const uint32_t fc = mp.r1;  // 2^32 mod p
    unsigned long long acc[NV];
    {
        // two-word accumulators, folded by 2^32 mod p every FOLDK products
        Acc2 ac[NV];
#pragma unroll
        for (int b = 0; b < NV; b++) ac[b] = Acc2{0u, 0u};
        if (slot < per) {
            // U rows in flight per thread.  GRAM: xh holds the weights in
            // Montgomery form, so mont_mul(xh[r], T[r][a]) = w_r T[r][a].
            constexpr int U = NV <= 8 ? 4 : (NV <= 16 ? 2 : 1);
            const int64_t stride = (int64_t)gridDim.x * per;
            int64_t r = (int64_t)blockIdx.x * per + slot;
            int cnt = 0;
            for (; r + (U - 1) * stride < N; r += U * stride) {
                uint32_t xs[U], tv[U][NV];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int64_t ru = r + u * stride;
                    xs[u] = GRAM ? mont_mul(__ldg(xh + ru), __ldg(t + ru * tstride + a), mp) : __ldg(xh + ru * m + a);
                    ldv<NV>(t + ru * tstride + yoff, tv[u]);
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
#pragma unroll
                    for (int b = 0; b < NV; b++) mac2(ac[b], xs[u], tv[u][b]);
                    if (++cnt == FOLDK) {
#pragma unroll
                        for (int b = 0; b < NV; b++) fold2w(ac[b], fc);
                        cnt = 0;
                    }
                }
            }
            for (; r < N; r += stride) {
                const uint32_t xv = GRAM ? mont_mul(__ldg(xh + r), __ldg(t + r * tstride + a), mp) : __ldg(xh + r * m + a);
                uint32_t tv[NV];
                ldv<NV>(t + r * tstride + yoff, tv);
#pragma unroll
                for (int b = 0; b < NV; b++) mac2(ac[b], xv, tv[b]);
                if (++cnt == FOLDK) {
#pragma unroll
                    for (int b = 0; b < NV; b++) fold2w(ac[b], fc);
                    cnt = 0;
                }
            }
        }
#pragma unroll
        for (int b = 0; b < NV; b++) acc[b] = red64(acc2_u64(ac[b]), mp);
    }
    if (pow2) {
        // lanes of a warp with the same a hold the same (a, b) entries:
        // butterfly over the slot bits (offsets m, 2m, ..., 16)
        for (int off = m; off < 32; off <<= 1)
#pragma unroll
            for (int b = 0; b < NV; b++) acc[b] += __shfl_xor_sync(0xffffffffu, acc[b], off);
        if (lane < m)
#pragma unroll
            for (int b = 0; b < NV; b++) red32[(warp * m + lane) * NV + b] = red64(acc[b], mp);
        __syncthreads();
        unsigned long long *dst = s_raw + (size_t)k_term * m * n;
        for (int e = tid; e < m * n; e += PROJ_THREADS) {
            const int aa = e / n, b = e % n;
            unsigned long long v = 0;
            for (int w = 0; w < PROJ_THREADS / 32; w++) v += red32[(w * m + aa) * NV + b];
            if (v) atomicAdd(dst + e, v);
        }
    } else {
        for (int i = tid; i < m * NV; i += PROJ_THREADS) red[i] = 0;
        __syncthreads();
        if (slot < per) {
#pragma unroll
            for (int b = 0; b < NV; b++)
                if (b < n && acc[b]) atomicAdd(&red[a * NV + b], acc[b]);
        }
        __syncthreads();
        unsigned long long *dst = s_raw + (size_t)k_term * m * n;
        for (int e = tid; e < m * n; e += PROJ_THREADS) {
            const unsigned long long v = red[(e / n) * NV + e % n];
            if (v) atomicAdd(dst + e, v);
        }
    }
}

__global__ void k_reduce_seq(int64_t count, const unsigned long long *__restrict__ s_raw,
                             uint32_t *__restrict__ S, ModP mp) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) S[i] = red64(s_raw[i], mp);
}

// random draws (tags: X 1, Y 2, D1 3, D2 4)
// map (locality-ordered matrix): entry i of the layout is index map[i] of
// the matrix as loaded, and the draw takes that index, so the sequence does
// not depend on the order (X^T A~^i Y is invariant under a simultaneous
// permutation of A~'s rows and columns, X and Y)
__global__ void k_derive_diag(uint64_t seed, uint64_t tag, int64_t len, uint32_t p,
                              uint32_t *__restrict__ out, const uint32_t *__restrict__ map) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) {
        const uint64_t gi = map ? (uint64_t)map[i] : (uint64_t)i;
        out[i] = (uint32_t)(1 + stream_hash(seed, tag, gi) % (uint64_t)(p - 1));
    }
}

// T0 = D1 Y (padded to nv columns with zeros; columns ycol0.. of a Y with
// ystride columns), d1sq = D1^2, and Xh = D1^{-1} X (X drawn with tag xtag,
// xwidth columns) or the Gram weights D1^{-2} (symmetric projection X = Y
// over the whole Y: S_2k = V_k^T V_k with T_k = D1 V_k; Montgomery form).
__global__ void k_prepare(int64_t N, int m, int n, int nv, uint64_t seed, uint64_t xtag, int xwidth, int ystride,
                          int ycol0, int gram, int paired, const uint32_t *__restrict__ d1, uint32_t *__restrict__ t0,
                          uint32_t *__restrict__ xh, uint32_t *__restrict__ d1sq, const uint32_t *__restrict__ nmap,
                          ModP mp, int trow) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint64_t gi = nmap ? (uint64_t)nmap[i] : (uint64_t)i;  // index of the draws
    const uint32_t d = d1[i];
    const uint32_t dinv = invm(d, mp);
    d1sq[i] = mulm(d, d, mp);
    // trow: row stride of t0 (0: the block's own width; a multi-job block is wider)
    const int tw = trow > 0 ? trow : (paired ? 2 * nv : nv), yo = paired ? nv : 0;
    for (int b = 0; b < nv; b++) {
        uint32_t yv = 0;
        if (b < n) yv = (uint32_t)(stream_hash(seed, TAG_Y, gi * ystride + ycol0 + b) % mp.p);
        t0[i * tw + yo + b] = mulm(d, yv, mp);
    }
    if (paired) {  // D1 X beside D1 Y, weights D1^{-2} for the cross Gram products
        for (int a = 0; a < nv; a++) {
            uint32_t xv = 0;
            if (a < m) xv = (uint32_t)(stream_hash(seed, xtag, gi * xwidth + a) % mp.p);
            t0[i * tw + a] = mulm(d, xv, mp);
        }
        xh[i] = to_mont(mulm(dinv, dinv, mp), mp);
        return;
    }
    if (gram) {
        xh[i] = to_mont(mulm(dinv, dinv, mp), mp);  // Montgomery form for the Gram projection
        return;
    }
    for (int a = 0; a < m; a++) {
        uint32_t xv = (uint32_t)(stream_hash(seed, xtag, gi * xwidth + a) % mp.p);
        xh[i * m + a] = mulm(dinv, xv, mp);
    }
}

// out = d^{-1} R mod p, elementwise (the Gram weights D2^{-1} of the odd terms of
// the symmetric projection: S_2k+1 = W^T D2^{-1} W with W = D2 A D1 V_k)
__global__ void k_inv_diag(int64_t len, const uint32_t *__restrict__ d, uint32_t *__restrict__ out, ModP mp) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] = to_mont(invm(d[i], mp), mp);  // Montgomery form for the Gram projection
}

// out (N x nv, padded) = D1 in (N x width)
// the caller's block is in the matrix's loaded order: row r of the layout
// reads (and writes back) row nmap[r] of it
__global__ void k_scale_pad(int64_t N, int width, int nv, const uint32_t *__restrict__ in,
                            const uint32_t *__restrict__ d1, uint32_t *__restrict__ out,
                            const uint32_t *__restrict__ nmap, ModP mp) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * nv) return;
    int64_t r = i / nv;
    int b = (int)(i % nv);
    const int64_t g = nmap ? (int64_t)nmap[r] : r;
    out[i] = b < width ? mulm(d1[r], in[g * width + b], mp) : 0;
}

__global__ void k_unpad(int64_t N, int width, int nv, const uint32_t *__restrict__ in,
                        uint32_t *__restrict__ out, const uint32_t *__restrict__ nmap) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * width) return;
    int64_t r = i / width;
    int b = (int)(i % width);
    const int64_t g = nmap ? (int64_t)nmap[r] : r;
    out[g * width + b] = in[r * nv + b];
}

// The iterated block in the matrix's row order, unscaled (T = D1 V): from the
// paired block [D1 A~^k X | D1 A~^k Y] the N x (m + n) block [A~^k X | A~^k Y],
// otherwise A~^k Y (N x n).
__global__ void k_export_state(int64_t N, int m, int n, int nv, int paired, const uint32_t *__restrict__ T,
                               const uint32_t *__restrict__ d1, uint32_t *__restrict__ out,
                               const uint32_t *__restrict__ nmap, ModP mp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t dinv = invm(d1[i], mp);
    const int64_t g = nmap ? (int64_t)nmap[i] : i;
    const int tw = paired ? 2 * nv : nv, w = paired ? m + n : n;
    if (paired) {
        for (int a = 0; a < m; a++) out[g * w + a] = mulm(dinv, T[i * tw + a], mp);
        for (int b = 0; b < n; b++) out[g * w + m + b] = mulm(dinv, T[i * tw + nv + b], mp);
    } else {
        for (int b = 0; b < n; b++) out[g * w + b] = mulm(dinv, T[i * tw + b], mp);
    }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <int NV, int WL>
void launch_spmm_kernel(wr_ctx *ctx, const SellView &A, const uint32_t *x, uint32_t *y, const uint32_t *scale,
                        unsigned long long *acc64, const ModP &mp, int *term_counter, bool cs,
                        const MultiEpi *me, int part) {
    const int64_t vblocks = (A.nseg + 7) / 8;
    const int64_t lblocks = (A.nchunks * Lanes<NV, WL>::G + 7) / 8;
    const int64_t blocks = std::max<int64_t>(vblocks + lblocks, term_counter ? 1 : 0);
    if (blocks <= 0) return;
    const MultiEpi one{};
#define WR_SPMM_LAUNCH(WIDEV, CSV, MULTIV)                                                                     \
    k_spmm<NV, WL, WIDEV, CSV, MULTIV><<<(unsigned)blocks, 256, 0, ctx->stream>>>(                             \
        A, x, y, scale, acc64, mp, term_counter, vblocks, me ? *me : one, part)
    if constexpr (NV >= 16) {
        if (me && me->jobs > 1) {
            if (A.wvals) {
                if (cs) WR_SPMM_LAUNCH(true, true, true); else WR_SPMM_LAUNCH(true, false, true);
            } else {
                if (cs) WR_SPMM_LAUNCH(false, true, true); else WR_SPMM_LAUNCH(false, false, true);
            }
            return;
        }
    }
    if (A.wvals) {
        if (cs) WR_SPMM_LAUNCH(true, true, false); else WR_SPMM_LAUNCH(true, false, false);
    } else {
        if (cs) WR_SPMM_LAUNCH(false, true, false); else WR_SPMM_LAUNCH(false, false, false);
    }
#undef WR_SPMM_LAUNCH
}

template <int NV>
wr_status launch_spmm_t(wr_ctx *ctx, const SellView &A, const uint32_t *x, uint32_t *y,
                        const uint32_t *scale, unsigned long long *acc64, const ModP &mp,
                        int *term_counter, int wl, bool cs, bool finalize, const MultiEpi *me, int part) {
    const int vblocks_any = (A.nseg + A.nchunks) > 0 || term_counter;
    switch (wl) {
        case 1:
            if constexpr (NV <= 32) { launch_spmm_kernel<NV, 1>(ctx, A, x, y, scale, acc64, mp, term_counter, cs, me, part); break; }
            else return fail(WR_EINVAL, "lane width too small for the block width");
        case 2:
            if constexpr (NV % 2 == 0) { launch_spmm_kernel<NV, 2>(ctx, A, x, y, scale, acc64, mp, term_counter, cs, me, part); break; }
            else return fail(WR_EINVAL, "lane width does not divide the block width");
        case 4:
            if constexpr (NV % 4 == 0) { launch_spmm_kernel<NV, 4>(ctx, A, x, y, scale, acc64, mp, term_counter, cs, me, part); break; }
            else return fail(WR_EINVAL, "lane width does not divide the block width");
        case 8:
            if constexpr (NV % 8 == 0) { launch_spmm_kernel<NV, 8>(ctx, A, x, y, scale, acc64, mp, term_counter, cs, me, part); break; }
            else return fail(WR_EINVAL, "lane width does not divide the block width");
        default: return fail(WR_EINVAL, "lane width must be 1, 2, 4 or 8");
    }
    if (vblocks_any) WR_LAUNCHED(ctx);
    if (finalize && A.nsplit > 0) {
        int64_t cnt = A.nsplit * NV;
        if (me && me->jobs > 1)
            k_finalize_split_multi<<<blocks_for(cnt, 256), 256, 0, ctx->stream>>>(A.nsplit, NV, A.split_row, acc64,
                                                                                 y, *me);
        else
            k_finalize_split<<<blocks_for(cnt, 256), 256, 0, ctx->stream>>>(A.nsplit, NV, A.split_row, acc64,
                                                                           y, scale, mp, part);
        WR_LAUNCHED(ctx);
    }
    return WR_OK;
}

// SpMM variant: residues per lane in the low bits (0 = the default for nv),
// SPMM_CS set for the streaming cache hints on entries and outputs
constexpr int SPMM_CS = 16;

// finalize = false leaves the split rows' sums in acc64 (used by the tuner only)
wr_status launch_spmm(wr_ctx *ctx, int nv, const SellView &A, const uint32_t *x, uint32_t *y,
                      const uint32_t *scale, unsigned long long *acc64, const ModP &mp,
                      int *term_counter, int variant = 0, bool finalize = true, const MultiEpi *me = nullptr,
                      int part = 0) {
    const bool cs = (variant & SPMM_CS) != 0;
    int wl = variant & (SPMM_CS - 1);
    if (wl <= 0 || wl > nv || nv / wl > 32) wl = default_lane_width(nv);
    switch (nv) {
        case 1: return launch_spmm_t<1>(ctx, A, x, y, scale, acc64, mp, term_counter, wl, cs, finalize, me, part);
        case 2: return launch_spmm_t<2>(ctx, A, x, y, scale, acc64, mp, term_counter, wl, cs, finalize, me, part);
        case 4: return launch_spmm_t<4>(ctx, A, x, y, scale, acc64, mp, term_counter, wl, cs, finalize, me, part);
        case 8: return launch_spmm_t<8>(ctx, A, x, y, scale, acc64, mp, term_counter, wl, cs, finalize, me, part);
        case 16: return launch_spmm_t<16>(ctx, A, x, y, scale, acc64, mp, term_counter, wl, cs, finalize, me, part);
        case 32: return launch_spmm_t<32>(ctx, A, x, y, scale, acc64, mp, term_counter, wl, cs, finalize, me, part);
        case 64: return launch_spmm_t<64>(ctx, A, x, y, scale, acc64, mp, term_counter, wl, cs, finalize, me, part);
        default: return fail(WR_EINVAL, "unsupported padded block width");
    }
}

// Lane-width tuner: times the candidate residues-per-lane (1, 2, 4, 8; at
// most 32 lanes per gathered row) of one SpMM layout on the matrix itself (zero block: the gather addresses, which
// set the time, do not depend on the values) and keeps the fastest.  The
// result never depends on the choice.
int nv_index(int nv) {
    int k = 0;
    while ((1 << k) < nv) k++;
    return k;
}

static wr_status tune_lane_width(wr_ctx *ctx, const Sell &S, int nv, int *out) {
    *out = default_lane_width(nv);
    if (S.nslots + S.nvent < (int64_t)1 << 20) return WR_OK;  // too small to matter
    cudaStream_t s = ctx->stream;
    DevBuf x, y, scale, acc;
    WR_TRY(dev_alloc(ctx, x, sizeof(uint32_t) * (size_t)std::max<int64_t>(S.ncols, 1) * nv));
    WR_TRY(dev_alloc(ctx, y, sizeof(uint32_t) * (size_t)std::max<int64_t>(S.nrows, 1) * nv));
    WR_TRY(dev_alloc(ctx, scale, sizeof(uint32_t) * (size_t)std::max<int64_t>(S.nrows, 1)));
    WR_TRY(dev_alloc(ctx, acc, sizeof(unsigned long long) * (size_t)std::max<int64_t>(S.nsplit, 1) * nv));
    WR_CUDA(cudaMemsetAsync(x.ptr, 0, x.bytes, s));
    WR_CUDA(cudaMemsetAsync(scale.ptr, 0, scale.bytes, s));
    WR_CUDA(cudaMemsetAsync(acc.ptr, 0, acc.bytes, s));
    const ModP mp = make_modp(2147483629u);
    const SellView v = view(S);
    cudaEvent_t e0, e1;
    WR_CUDA(cudaEventCreate(&e0));
    WR_CUDA(cudaEventCreate(&e1));
    float best = 0.0f;
    for (int cs : {0, SPMM_CS})
        for (int wl : {1, 2, 4, 8}) {
            if (wl > nv || nv % wl != 0 || nv / wl > 32) continue;
            for (int w = 0; w < 2; w++)
                WR_TRY(launch_spmm(ctx, nv, v, x.as<uint32_t>(), y.as<uint32_t>(), scale.as<uint32_t>(),
                                   acc.as<unsigned long long>(), mp, nullptr, wl | cs, false));
            WR_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < 5; r++)
                WR_TRY(launch_spmm(ctx, nv, v, x.as<uint32_t>(), y.as<uint32_t>(), scale.as<uint32_t>(),
                                   acc.as<unsigned long long>(), mp, nullptr, wl | cs, false));
            WR_CUDA(cudaEventRecord(e1, s));
            WR_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best == 0.0f || ms < best) {
                best = ms;
                *out = wl | cs;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return WR_OK;
}

// the lane width for a layout: forced by the context, else tuned once per
// matrix, layout and block width (when the context tunes), else the default
static wr_status lane_width_for(wr_ctx *ctx, const wr_matrix *mat, const Sell &S, int nv, int *out) {
    const int lw = ctx->lane_width & 15;
    if (lw > 0 && lw <= nv && nv % lw == 0 && nv / lw <= 32) {
        *out = ctx->lane_width;
        return WR_OK;
    }
    if (!ctx->autotune) {
        *out = default_lane_width(nv);
        return WR_OK;
    }
    const int layout = &S == &mat->a ? 0 : 1, k = nv_index(nv);
    std::lock_guard<std::mutex> lk(mat->tune_mu);
    if (mat->tuned_w[layout][k] == 0) {
        int w = 0;
        WR_TRY(tune_lane_width(ctx, S, nv, &w));
        mat->tuned_w[layout][k] = w;
    }
    *out = mat->tuned_w[layout][k];
    return WR_OK;
}

}  // namespace

wr_status launch_spmm_multi(wr_ctx *ctx, int nv, const SellView &A, const uint32_t *x, uint32_t *y,
                            unsigned long long *acc64, const MultiEpi &me, int *term_counter, int variant) {
    if (me.jobs < 2 || me.jobs > MULTI_MAX_JOBS || nv < 16 || (me.jobs << me.jw_log) > nv)
        return fail(WR_EINVAL, "multi-job SpMM: 2..4 jobs over a block of 16 columns or more");
    return launch_spmm(ctx, nv, A, x, y, nullptr, acc64, me.mp[0], term_counter, variant, true, &me);
}

wr_status spmm_variant_for(wr_ctx *ctx, const wr_matrix *mat, const Sell &S, int nv, int *out) {
    return lane_width_for(ctx, mat, S, nv, out);
}

namespace {

template <int NV, bool GRAM>
void launch_project_t(wr_ctx *ctx, unsigned grid, int64_t N, int m, int n, const uint32_t *xh,
                      const uint32_t *t, unsigned long long *s_raw, const int *term_counter, int tmul, int toff,
                      int64_t L, int tstride, int yoff, const ModP &mp) {
    if (tstride <= 0) tstride = NV;
    if (mp.lazy >= 16)  // p < 2^30
        k_project<NV, 14, GRAM><<<grid, PROJ_THREADS, 0, ctx->stream>>>(N, m, n, xh, t, s_raw, term_counter, tmul,
                                                                         toff, L, tstride, yoff, mp);
    else
        k_project<NV, 2, GRAM><<<grid, PROJ_THREADS, 0, ctx->stream>>>(N, m, n, xh, t, s_raw, term_counter, tmul,
                                                                        toff, L, tstride, yoff, mp);
}

// gram = false: S_raw[k] += xh^T t (xh: N x m).  gram = true: S_raw[k] +=
// sum_r xh[r] t[r]^T t[r] (xh: N weights, m = n).  k = tmul * counter + toff.
wr_status launch_project(wr_ctx *ctx, int64_t N, int m, int n, int nv, const uint32_t *xh,
                         const uint32_t *t, unsigned long long *s_raw, const int *term_counter,
                         const ModP &mp, bool gram = false, int tmul = 1, int toff = 0,
                         int64_t L = INT64_MAX, int tstride = 0, int yoff = 0) {
    const int per = PROJ_THREADS / m;
    const int64_t need = std::max<int64_t>((N + per - 1) / per, 1);
    const unsigned grid = (unsigned)std::min<int64_t>(need, (int64_t)ctx->num_sms * 2);
#define WR_PROJ_CASE(NVV)                                                                                    \
    case NVV:                                                                                                \
        if (gram)                                                                                            \
            launch_project_t<NVV, true>(ctx, grid, N, m, n, xh, t, s_raw, term_counter, tmul, toff, L, tstride, yoff, mp); \
        else                                                                                                 \
            launch_project_t<NVV, false>(ctx, grid, N, m, n, xh, t, s_raw, term_counter, tmul, toff, L, tstride, yoff, mp); \
        break;
    switch (nv) {
        WR_PROJ_CASE(1)
        WR_PROJ_CASE(2)
        WR_PROJ_CASE(4)
        WR_PROJ_CASE(8)
        WR_PROJ_CASE(16)
        WR_PROJ_CASE(32)
        default: return fail(WR_EINVAL, "unsupported padded block width");
    }
#undef WR_PROJ_CASE
    WR_LAUNCHED(ctx);
    return WR_OK;
}

}  // namespace

// State of one sequence run (device buffers), shared by wr_rank and the
// step-level entry points.
struct SeqState {
    Resolved r;
    ModP mp;
    const Sell *first = nullptr;   // pass 1 layout (output in the other space)
    const Sell *second = nullptr;  // pass 2 layout (output in N-space)
    int wl1 = 0, wl2 = 0;          // residues per lane of the two passes
    // column slabs of the two passes (empty: one launch over the whole layout)
    const std::vector<Sell> *slabs1 = nullptr, *slabs2 = nullptr;
    DevBuf T, Wb, D1, D2, d1sq, xh, w2, acc1, acc2, s_raw, counter, err;
    // The two Gram projections of an application beside the passes
    // (symmetric and paired projections, wr_set_projection_overlap): they run
    // on a side stream, forked after the pass whose output they read and
    // joined before the pass that overwrites it, so the Gram of W_k runs
    // beside pass 2 and the Gram of T_k beside pass 1 of the next
    // application; all of a group's work joins the sequence stream at its end.
    // The side stream keeps its own term counter (gcounter = application + 1,
    // advanced after each application's second Gram).
    cudaStream_t side = nullptr;
    cudaEvent_t ev_p1 = nullptr, ev_p2 = nullptr, ev_g1 = nullptr, ev_g2 = nullptr;
    bool g1_pending = false, g2_pending = false;
    DevBuf gcounter;
    SeqState() = default;
    SeqState(const SeqState &) = delete;
    SeqState &operator=(const SeqState &) = delete;
    ~SeqState() {
        for (cudaEvent_t e : {ev_p1, ev_p2, ev_g1, ev_g2})
            if (e) cudaEventDestroy(e);
        if (side) cudaStreamDestroy(side);
    }
};

__global__ void k_bump(int *__restrict__ c) { *c += 1; }

// ctx->stream switched to another stream for the launches of one scope
struct StreamSwap {
    wr_ctx *ctx;
    cudaStream_t keep;
    StreamSwap(wr_ctx *c, cudaStream_t s) : ctx(c), keep(c->stream) { c->stream = s; }
    ~StreamSwap() { ctx->stream = keep; }
};

// Column slabs (off unless the context sets a slab size, ctx->slab_bytes > 0):
// a pass whose gathered block is larger than the slab size runs as S launches
// over column ranges of the matrix, S = ceil(block bytes / slab size), so
// that the block rows one launch gathers stay in L2; the output rows carry
// residues from one launch to the next (k_spmm's part argument).  The layouts
// are built from the CSR kept with the matrix on first use.  Measured on the
// 1.9M x 1.95M matrix at width 64 they are slower (a pass 1.48 ms without,
// 2.1-5.3 ms with 4-16 slabs): every slab reads and writes all output rows.
constexpr int SLAB_MAX = 64;

static wr_status slabs_for(wr_ctx *ctx, const wr_matrix *mat, const Sell &S, int nv,
                           const std::vector<Sell> **out) {
    *out = nullptr;
    if (ctx->slab_bytes <= 0 || !mat->csr_rp[0].ptr) return WR_OK;
    const int64_t target = ctx->slab_bytes;
    const int64_t block = S.ncols * (int64_t)nv * 4;
    if (block <= target || S.ncols < 2) return WR_OK;
    const int n = (int)std::min<int64_t>(std::min<int64_t>((block + target - 1) / target, SLAB_MAX), S.ncols);
    const int layout = &S == &mat->a ? 0 : 1;
    std::lock_guard<std::mutex> lk(mat->tune_mu);
    if (mat->slab_n[layout] != n) {
        std::vector<Sell> v(n);
        const int64_t width = (S.ncols + n - 1) / n;
        for (int s = 0; s < n; s++) {
            const int64_t c0 = std::min<int64_t>(s * width, S.ncols), c1 = std::min<int64_t>(c0 + width, S.ncols);
            WR_TRY(build_sell_slab(ctx, S.nrows, S.ncols, mat->csr_rp[layout].as<int64_t>(),
                                   mat->csr_ci[layout].as<int32_t>(), mat->csr_va[layout].as<int32_t>(), (int32_t)c0,
                                   (int32_t)c1, v[s], mat->wide));
        }
        mat->slabs[layout] = std::move(v);
        mat->slab_n[layout] = n;
    }
    *out = &mat->slabs[layout];
    return WR_OK;
}

// one pass over the whole layout, or over its column slabs
static wr_status launch_pass(wr_ctx *ctx, int nv, const Sell &S, const std::vector<Sell> *slabs, const uint32_t *x,
                             uint32_t *y, const uint32_t *scale, unsigned long long *acc64, const ModP &mp,
                             int *term_counter, int variant) {
    if (!slabs || slabs->size() < 2)
        return launch_spmm(ctx, nv, view(S), x, y, scale, acc64, mp, term_counter, variant);
    const int n = (int)slabs->size();
    for (int s = 0; s < n; s++)
        WR_TRY(launch_spmm(ctx, nv, view((*slabs)[s]), x, y, scale, acc64, mp, s == 0 ? term_counter : nullptr,
                           variant, true, nullptr, s == 0 ? 1 : (s == n - 1 ? 3 : 2)));
    return WR_OK;
}

static int64_t max_split(const Sell &S, const std::vector<Sell> *slabs) {
    int64_t m = S.nsplit;
    if (slabs)
        for (const auto &x : *slabs) m = std::max<int64_t>(m, x.nsplit);
    return m;
}

// A Gram projection S_raw[tmul * counter + toff] += sum_r w_r t[r][0..m)^T
// t[r][yoff..yoff+n): on the tensor cores (bf16 digit products, exact) when
// the context asks for them, or automatically for blocks of 16 columns and
// more; otherwise with 64-bit integer multiply-adds.  Same result either way.
static bool use_tc_gram(const wr_ctx *ctx, int m, int n, int tstride, int yoff) {
    if (ctx->tensor_proj == 0 || !gram_tc_supported(m, n, tstride, yoff)) return false;
    return ctx->tensor_proj == 1 || (m >= 16 && n >= 16);
}

static wr_status launch_gram_to(wr_ctx *ctx, const Resolved &r, const ModP &mp, int64_t rows, const uint32_t *w,
                                const uint32_t *t, int tmul, int toff, int tstride, int yoff,
                                unsigned long long *s_raw, const int *counter, int *err) {
    if (use_tc_gram(ctx, r.m, r.n, tstride, yoff))
        return launch_gram_tc(ctx, rows, r.m, r.n, w, t, tstride, yoff, s_raw, counter, tmul, toff, r.L, mp, err);
    return launch_project(ctx, rows, r.m, r.n, r.nv, w, t, s_raw, counter, mp, true, tmul, toff, r.L, tstride, yoff);
}

static wr_status launch_gram(wr_ctx *ctx, SeqState &st, int64_t rows, const uint32_t *w, const uint32_t *t,
                             int tmul, int toff, int tstride, int yoff, const int *counter = nullptr) {
    return launch_gram_to(ctx, st.r, st.mp, rows, w, t, tmul, toff, tstride, yoff, st.s_raw.as<unsigned long long>(),
                          counter ? counter : st.counter.as<int>(), st.err.as<int>());
}

static wr_status seq_setup(wr_ctx *ctx, const wr_matrix *mat, const Resolved &r, SeqState &st,
                           bool want_projection) {
    st.r = r;
    st.mp = make_modp(r.p);
    st.first = r.side == 0 ? &mat->a : &mat->at;
    st.second = r.side == 0 ? &mat->at : &mat->a;
    const int nv = r.nvs;  // SpMM width (2 nv for the paired generic block)
    WR_TRY(lane_width_for(ctx, mat, *st.first, nv, &st.wl1));
    WR_TRY(lane_width_for(ctx, mat, *st.second, nv, &st.wl2));
    WR_TRY(slabs_for(ctx, mat, *st.first, nv, &st.slabs1));
    WR_TRY(slabs_for(ctx, mat, *st.second, nv, &st.slabs2));
    WR_TRY(dev_alloc(ctx, st.T, sizeof(uint32_t) * std::max<int64_t>(r.N * nv, 1)));
    WR_TRY(dev_alloc(ctx, st.Wb, sizeof(uint32_t) * std::max<int64_t>(r.M * nv, 1)));
    WR_TRY(dev_alloc(ctx, st.D1, sizeof(uint32_t) * std::max<int64_t>(r.N, 1)));
    WR_TRY(dev_alloc(ctx, st.D2, sizeof(uint32_t) * std::max<int64_t>(r.M, 1)));
    WR_TRY(dev_alloc(ctx, st.d1sq, sizeof(uint32_t) * std::max<int64_t>(r.N, 1)));
    WR_TRY(dev_alloc(ctx, st.xh, sizeof(uint32_t) * std::max<int64_t>(r.N * r.m, 1)));
    WR_TRY(dev_alloc(ctx, st.acc1,
                     sizeof(unsigned long long) * std::max<int64_t>(max_split(*st.first, st.slabs1) * nv, 1)));
    WR_TRY(dev_alloc(ctx, st.acc2,
                     sizeof(unsigned long long) * std::max<int64_t>(max_split(*st.second, st.slabs2) * nv, 1)));
    WR_TRY(dev_alloc(ctx, st.counter, sizeof(int)));
    WR_TRY(dev_alloc(ctx, st.err, sizeof(int)));
    cudaStream_t s = ctx->stream;
    WR_CUDA(cudaMemsetAsync(st.err.ptr, 0, sizeof(int), s));
    WR_CUDA(cudaMemsetAsync(st.acc1.ptr, 0, st.acc1.bytes, s));
    WR_CUDA(cudaMemsetAsync(st.acc2.ptr, 0, st.acc2.bytes, s));
    WR_CUDA(cudaMemsetAsync(st.counter.ptr, 0, sizeof(int), s));
    if (want_projection && ctx->proj_overlap && (r.gram || r.paired)) {
        int prio = 0;
        WR_CUDA(cudaStreamGetPriority(s, &prio));
        WR_CUDA(cudaStreamCreateWithPriority(&st.side, cudaStreamNonBlocking, prio));
        for (cudaEvent_t *e : {&st.ev_p1, &st.ev_p2, &st.ev_g1, &st.ev_g2})
            WR_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        WR_TRY(dev_alloc(ctx, st.gcounter, sizeof(int)));
        WR_CUDA(cudaMemsetAsync(st.gcounter.ptr, 0, sizeof(int), s));
        k_bump<<<1, 1, 0, s>>>(st.gcounter.as<int>());  // the first application's terms: counter 1
        WR_LAUNCHED(ctx);
    }
    if (r.N > 0) {
        k_derive_diag<<<blocks_for(r.N, 256), 256, 0, s>>>(r.seed, TAG_D1, r.N, r.p, st.D1.as<uint32_t>(), r.nmap);
        WR_LAUNCHED(ctx);
    }
    if (r.M > 0) {
        k_derive_diag<<<blocks_for(r.M, 256), 256, 0, s>>>(r.seed, TAG_D2, r.M, r.p, st.D2.as<uint32_t>(), r.mmap);
        WR_LAUNCHED(ctx);
    }
    if (want_projection && r.N > 0) {
        k_prepare<<<blocks_for(r.N, 128), 128, 0, s>>>(r.N, r.m, r.n, r.nv, r.seed, r.xtag, r.xwidth, r.ystride,
                                                      r.ycol0, r.gram ? 1 : 0, r.paired ? 1 : 0, st.D1.as<uint32_t>(),
                                                      st.T.as<uint32_t>(), st.xh.as<uint32_t>(),
                                                      st.d1sq.as<uint32_t>(), r.nmap, st.mp, 0);
        WR_LAUNCHED(ctx);
    }
    if (want_projection && (r.gram || r.paired) && r.M > 0) {
        WR_TRY(dev_alloc(ctx, st.w2, sizeof(uint32_t) * r.M));
        k_inv_diag<<<blocks_for(r.M, 256), 256, 0, s>>>(r.M, st.D2.as<uint32_t>(), st.w2.as<uint32_t>(), st.mp);
        WR_LAUNCHED(ctx);
    }
    return WR_OK;
}

// Terms produced by k black-box applications: one each (generic projection),
// two each with the symmetric projection, where Ã = D1 A^T D2 A D1 is
// symmetric and V_k = Ã^k Y gives S_2k = V_k^T V_k and
// S_2k+1 = (A D1 V_k)^T D2 (A D1 V_k).
static int64_t seq_applications(const Resolved &r, int64_t L) {
    const int64_t terms = std::max<int64_t>(L - 1, 0);
    return (r.gram || r.paired) ? (terms + 1) / 2 : terms;
}

// One iteration: W = D2 A T, T <- D1^2 A^T W (or the rows-side analogue),
// then the projections: the new T into S_raw[counter] (generic), or W and the
// new T into S_raw[2 counter - 1] and S_raw[2 counter] (symmetric; terms past
// L - 1 are skipped).
static wr_status seq_iteration(wr_ctx *ctx, SeqState &st, cudaEvent_t *ev) {
    const int nv = st.r.nvs;
    cudaStream_t s = ctx->stream;
    if (st.side) {
        const int ts = nv, yo = st.r.paired ? st.r.nv : 0;
        if (ev) WR_CUDA(cudaEventRecord(ev[0], s));
        if (st.g1_pending) WR_CUDA(cudaStreamWaitEvent(s, st.ev_g1, 0));  // pass 1 overwrites W
        WR_TRY(launch_pass(ctx, nv, *st.first, st.slabs1, st.T.as<uint32_t>(), st.Wb.as<uint32_t>(),
                           st.D2.as<uint32_t>(), st.acc1.as<unsigned long long>(), st.mp, st.counter.as<int>(), st.wl1));
        if (ev) WR_CUDA(cudaEventRecord(ev[1], s));
        WR_CUDA(cudaEventRecord(st.ev_p1, s));
        {
            StreamSwap sw(ctx, st.side);
            WR_CUDA(cudaStreamWaitEvent(st.side, st.ev_p1, 0));
            WR_TRY(launch_gram(ctx, st, st.r.M, st.w2.as<uint32_t>(), st.Wb.as<uint32_t>(), 2, -1, ts, yo,
                               st.gcounter.as<int>()));
            WR_CUDA(cudaEventRecord(st.ev_g1, st.side));
        }
        st.g1_pending = true;
        if (st.g2_pending) WR_CUDA(cudaStreamWaitEvent(s, st.ev_g2, 0));  // pass 2 overwrites T
        WR_TRY(launch_pass(ctx, nv, *st.second, st.slabs2, st.Wb.as<uint32_t>(), st.T.as<uint32_t>(),
                           st.d1sq.as<uint32_t>(), st.acc2.as<unsigned long long>(), st.mp, nullptr, st.wl2));
        if (ev) WR_CUDA(cudaEventRecord(ev[2], s));
        WR_CUDA(cudaEventRecord(st.ev_p2, s));
        {
            StreamSwap sw(ctx, st.side);
            WR_CUDA(cudaStreamWaitEvent(st.side, st.ev_p2, 0));
            WR_TRY(launch_gram(ctx, st, st.r.N, st.xh.as<uint32_t>(), st.T.as<uint32_t>(), 2, 0, ts, yo,
                               st.gcounter.as<int>()));
            k_bump<<<1, 1, 0, st.side>>>(st.gcounter.as<int>());
            WR_LAUNCHED(ctx);
            WR_CUDA(cudaEventRecord(st.ev_g2, st.side));
        }
        st.g2_pending = true;
        return WR_OK;
    }
    if (ev) WR_CUDA(cudaEventRecord(ev[0], ctx->stream));
    WR_TRY(launch_pass(ctx, nv, *st.first, st.slabs1, st.T.as<uint32_t>(), st.Wb.as<uint32_t>(), st.D2.as<uint32_t>(),
                       st.acc1.as<unsigned long long>(), st.mp, st.counter.as<int>(), st.wl1));
    if (ev) WR_CUDA(cudaEventRecord(ev[1], ctx->stream));
    WR_TRY(launch_pass(ctx, nv, *st.second, st.slabs2, st.Wb.as<uint32_t>(), st.T.as<uint32_t>(),
                       st.d1sq.as<uint32_t>(), st.acc2.as<unsigned long long>(), st.mp, nullptr, st.wl2));
    if (ev) WR_CUDA(cudaEventRecord(ev[2], ctx->stream));
    if (st.r.gram || st.r.paired) {
        const int ts = nv, yo = st.r.paired ? st.r.nv : 0;
        WR_TRY(launch_gram(ctx, st, st.r.M, st.w2.as<uint32_t>(), st.Wb.as<uint32_t>(), 2, -1, ts, yo));
        WR_TRY(launch_gram(ctx, st, st.r.N, st.xh.as<uint32_t>(), st.T.as<uint32_t>(), 2, 0, ts, yo));
    } else {
        WR_TRY(launch_project(ctx, st.r.N, st.r.m, st.r.n, nv, st.xh.as<uint32_t>(), st.T.as<uint32_t>(),
                              st.s_raw.as<unsigned long long>(), st.counter.as<int>(), st.mp, false, 1, 0,
                              st.r.L));
    }
    return WR_OK;
}

// The side stream's Gram projections joined into the sequence stream (end of
// a group of applications: its terms are complete after this point).
static wr_status seq_join(wr_ctx *ctx, SeqState &st) {
    if (st.side && st.g2_pending) WR_CUDA(cudaStreamWaitEvent(ctx->stream, st.ev_g2, 0));
    st.g1_pending = st.g2_pending = false;
    return WR_OK;
}

static double spmm_pass_bytes(const Sell &s, int nv, int64_t nnz) {
    // packed entries (4 B each), gathered block read once, output written
    // once, one scale residue per output row
    return 4.0 * (double)nnz + 4.0 * nv * (double)(s.ncols + s.nrows) + 4.0 * (double)s.nrows;
}

// generic projection with m = n: A~ is symmetric, so with U_k = A~^k X and
// V_k = A~^k Y, S_2k = U_k^T V_k and S_2k+1 = (A D1 U_k)^T D2 (A D1 V_k);
// X and Y ride in one block of twice the width (up to 64 residues per row),
// two terms per application
bool pairs_generic(const wr_ctx *ctx, const Resolved &r) {
    return !r.symmetric && r.m == r.n && 2 * r.nv <= 64 && ctx->pair_generic;
}

wr_status run_sequence(wr_ctx *ctx, const wr_matrix *mat, const wr_params &prm, int64_t L,
                       uint32_t *d_S, double *setup_ms, double *seq_ms, SeqFeed *feed, StateOut *out) {
    Resolved r;
    WR_TRY(resolve(mat, &prm, r));
    if (pairs_generic(ctx, r)) {
        r.paired = true;
        r.nvs = 2 * r.nv;
    }
    return run_sequence_resolved(ctx, mat, r, L, d_S, setup_ms, seq_ms, feed, out);
}

// Terms final after `done` applications (the initial projection gives S_0).
static int64_t terms_ready(const Resolved &r, int64_t done, int64_t L) {
    return std::min<int64_t>((r.gram || r.paired) ? 2 * done + 1 : done + 1, L);
}

// Fed mode: reduce the terms [from, to) into d_S and publish an event after them.
static wr_status publish_terms(wr_ctx *ctx, SeqState &st, int64_t from, int64_t to, uint32_t *d_S,
                               SeqFeed *feed) {
    const int64_t E = (int64_t)st.r.m * st.r.n;
    if (to > from) {
        k_reduce_seq<<<blocks_for((to - from) * E, 256), 256, 0, ctx->stream>>>(
            (to - from) * E, st.s_raw.as<unsigned long long>() + from * E, d_S + from * E, st.mp);
        WR_LAUNCHED(ctx);
    }
    cudaEvent_t ev;
    WR_CUDA(cudaEventCreateWithFlags(&ev, WAIT_EVENT_FLAGS));
    cudaError_t ce = cudaEventRecord(ev, ctx->stream);
    {
        std::lock_guard<std::mutex> lk(feed->mu);
        feed->ev.push_back(ev);  // the feed's owner destroys it
        feed->ready.push_back(ce == cudaSuccess ? to : -1);
    }
    feed->cv.notify_all();
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaEventRecord");
    return WR_OK;
}

static wr_status export_state(wr_ctx *ctx, const SeqState &st, uint32_t *dst) {
    if (!dst || st.r.N <= 0) return WR_OK;
    k_export_state<<<blocks_for(st.r.N, 128), 128, 0, ctx->stream>>>(st.r.N, st.r.m, st.r.n, st.r.nv,
                                                                      st.r.paired ? 1 : 0, st.T.as<uint32_t>(),
                                                                      st.D1.as<uint32_t>(), dst, st.r.nmap, st.mp);
    WR_LAUNCHED(ctx);
    return WR_OK;
}

wr_status run_sequence_resolved(wr_ctx *ctx, const wr_matrix *mat, Resolved r, int64_t L, uint32_t *d_S,
                                double *setup_ms, double *seq_ms, SeqFeed *feed, StateOut *out) {
    r.L = L;
    cudaStream_t s = ctx->stream;
    cudaEvent_t e0, e1, e2;
    WR_CUDA(cudaEventCreate(&e0));
    WR_CUDA(cudaEventCreate(&e1));
    WR_CUDA(cudaEventCreateWithFlags(&e2, cudaEventBlockingSync));  // waited on below, asleep
    WR_CUDA(cudaEventRecord(e0, s));
    SeqState st;
    WR_TRY(seq_setup(ctx, mat, r, st, true));
    const int64_t E = (int64_t)r.m * r.n;
    WR_TRY(dev_alloc(ctx, st.s_raw, sizeof(unsigned long long) * std::max<int64_t>(L * E, 1)));
    WR_CUDA(cudaMemsetAsync(st.s_raw.ptr, 0, st.s_raw.bytes, s));
    if (L > 0) {
        if (r.gram || r.paired)
            WR_TRY(launch_gram(ctx, st, r.N, st.xh.as<uint32_t>(), st.T.as<uint32_t>(), 2, 0, r.nvs,
                               r.paired ? r.nv : 0));
        else
            WR_TRY(launch_project(ctx, r.N, r.m, r.n, r.nv, st.xh.as<uint32_t>(), st.T.as<uint32_t>(),
                                  st.s_raw.as<unsigned long long>(), st.counter.as<int>(), st.mp, false, 1, 0, L,
                                  r.nvs, 0));
    }
    if (out && out->snap_at == 0) WR_TRY(export_state(ctx, st, out->d_snap));
    int64_t published = 0;
    if (feed) {
        WR_TRY(publish_terms(ctx, st, 0, terms_ready(r, 0, L), d_S, feed));
        published = terms_ready(r, 0, L);
    }
    WR_CUDA(cudaEventRecord(e1, s));

    // profiling: every PROF_EVERY-th group of iterations is launched eagerly
    // with CUDA events around the two SpMM passes
    const int64_t iters = seq_applications(r, L);
    const int64_t G = 64;
    const int PROF_EVERY = 8;
    std::vector<cudaEvent_t> pev;
    if (ctx->profiling) {
        pev.resize(3 * G);
        for (auto &e : pev) WR_CUDA(cudaEventCreate(&e));
    }
    double prof_ms = 0.0;
    int64_t prof_launches = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int64_t graph_launches = 0;  // kernel nodes in one replay
    if (iters >= G) {
        const int64_t before = ctx->launches;
        WR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        wr_status cst = WR_OK;
        for (int64_t i = 0; i < G && cst == WR_OK; i++) cst = seq_iteration(ctx, st, nullptr);
        if (cst == WR_OK) cst = seq_join(ctx, st);
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        st.g1_pending = st.g2_pending = false;
        graph_launches = ctx->launches - before;
        ctx->launches = before;
        if (cst != WR_OK) { if (graph) cudaGraphDestroy(graph); return cst; }
        WR_CUDA(ce);
        WR_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    }
    int64_t done = 0, group = 0;
    wr_status loop_st = WR_OK;
    while (done < iters && loop_st == WR_OK) {
        if (feed && feed->throttle > 0) {
            // early termination: stop once the consumer has enough terms, and
            // keep few groups in flight so that its decision arrives in time
            if (published >= feed->stop_at.load()) break;
            const int64_t w = (int64_t)feed->ev.size() - feed->throttle;  // this thread alone appends
            if (w >= 0) {
                cudaError_t ce = cudaEventSynchronize(feed->ev[w]);
                if (ce != cudaSuccess) { loop_st = cuda_fail(ce, "cudaEventSynchronize"); break; }
            }
            if (published >= feed->stop_at.load()) break;
        }
        // a snapshot of the block ends the group at its application count
        const int64_t lim = (out && out->d_snap && out->snap_at > done) ? std::min(out->snap_at, iters) : iters;
        const int64_t todo = std::min(G, lim - done);
        if (todo == G && exec && !(ctx->profiling && group % PROF_EVERY == 0)) {
            cudaError_t ce = cudaGraphLaunch(exec, s);
            if (ce != cudaSuccess) loop_st = cuda_fail(ce, "cudaGraphLaunch");
            ctx->launches += graph_launches;
        } else {
            const bool prof = ctx->profiling;
            for (int64_t i = 0; i < todo && loop_st == WR_OK; i++)
                loop_st = seq_iteration(ctx, st, prof ? &pev[3 * i] : nullptr);
            if (loop_st == WR_OK) loop_st = seq_join(ctx, st);
            if (prof && loop_st == WR_OK) {
                cudaError_t ce = cudaEventSynchronize(pev[3 * (todo - 1) + 2]);
                if (ce != cudaSuccess) loop_st = cuda_fail(ce, "cudaEventSynchronize");
                for (int64_t i = 0; i < todo && loop_st == WR_OK; i++) {
                    float a = 0, b = 0;
                    cudaEventElapsedTime(&a, pev[3 * i], pev[3 * i + 1]);
                    cudaEventElapsedTime(&b, pev[3 * i + 1], pev[3 * i + 2]);
                    prof_ms += a + b;
                    prof_launches += 2;
                    ctx->last.spmm_bytes += spmm_pass_bytes(*st.first, r.nvs, mat->nnz) +
                                            spmm_pass_bytes(*st.second, r.nvs, mat->nnz);
                }
            }
        }
        done += todo;
        group++;
        if (out && out->d_snap && done == out->snap_at && loop_st == WR_OK) loop_st = export_state(ctx, st, out->d_snap);
        if (feed && loop_st == WR_OK) {
            const int64_t t = terms_ready(r, done, L);
            loop_st = publish_terms(ctx, st, published, t, d_S, feed);
            published = t;
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto &e : pev) cudaEventDestroy(e);
    WR_TRY(loop_st);
    if (out) {
        WR_TRY(export_state(ctx, st, out->d_last));
        out->applications = done;
        out->paired = r.paired;
    }
    if (!feed && L * E > 0) {
        k_reduce_seq<<<blocks_for(L * E, 256), 256, 0, s>>>(L * E, st.s_raw.as<unsigned long long>(), d_S,
                                                           st.mp);
        WR_LAUNCHED(ctx);
    }
    int herr = 0;
    WR_CUDA(cudaMemcpyAsync(&herr, st.err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaEventRecord(e2, s));
    WR_CUDA(cudaEventSynchronize(e2));
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, e0, e1);
    cudaEventElapsedTime(&b, e1, e2);
    if (herr) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        return fail(WR_ETIMEDOUT, "tensor-core projection: a bounded wait ran out");
    }
    if (setup_ms) *setup_ms = a;
    if (seq_ms) *seq_ms = b;
    ctx->last.sequence_terms = feed ? published : L;
    ctx->last.spmm_ms += prof_ms;
    ctx->last.spmm_launches += prof_launches;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    return WR_OK;
}

__global__ void k_to_mont_vec(int64_t len, const uint32_t *__restrict__ in, uint32_t *__restrict__ out, ModP mp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] = to_mont(in[i], mp);
}

// G (m x n) = sum_r w_r t[r][0..m)^T t[r][yoff..yoff+n) mod p, through the
// same kernels as the sequence's Gram projections
wr_status gram_device(wr_ctx *ctx, uint32_t p, int64_t N, int m, int n, const uint32_t *t, int tstride, int yoff,
                      const uint32_t *w, uint32_t *G) {
    if (m < 1 || m > 32 || n < 1 || n > 32) return fail(WR_EINVAL, "m and n must be in 1..32");
    const int nv = padded_width(n);
    if (N < 0 || tstride < m || yoff < 0 || yoff % nv != 0 || tstride % nv != 0 || yoff + nv > tstride)
        return fail(WR_EINVAL, "rows of t: tstride residues, a multiple of the padded width nv >= m and >= yoff + nv, "
                               "yoff a multiple of nv");
    if (reinterpret_cast<uintptr_t>(t) % 16 != 0) return fail(WR_EINVAL, "t must be 16-byte aligned");
    SeqState st;
    st.mp = make_modp(p);
    st.r.m = m;
    st.r.n = n;
    st.r.nv = nv;
    st.r.L = 1;
    cudaStream_t s = ctx->stream;
    DevBuf wm;
    WR_TRY(dev_alloc(ctx, wm, sizeof(uint32_t) * std::max<int64_t>(N, 1)));
    WR_TRY(dev_alloc(ctx, st.s_raw, sizeof(unsigned long long) * m * n));
    WR_TRY(dev_alloc(ctx, st.counter, sizeof(int)));
    WR_TRY(dev_alloc(ctx, st.err, sizeof(int)));
    WR_CUDA(cudaMemsetAsync(st.s_raw.ptr, 0, st.s_raw.bytes, s));
    WR_CUDA(cudaMemsetAsync(st.counter.ptr, 0, sizeof(int), s));
    WR_CUDA(cudaMemsetAsync(st.err.ptr, 0, sizeof(int), s));
    if (N > 0) {
        k_to_mont_vec<<<blocks_for(N, 256), 256, 0, s>>>(N, w, wm.as<uint32_t>(), st.mp);
        WR_LAUNCHED(ctx);
        WR_TRY(launch_gram(ctx, st, N, wm.as<uint32_t>(), t, 1, 0, tstride, yoff));
    }
    k_reduce_seq<<<blocks_for((int64_t)m * n, 256), 256, 0, s>>>((int64_t)m * n, st.s_raw.as<unsigned long long>(),
                                                                G, st.mp);
    WR_LAUNCHED(ctx);
    int herr = 0;
    WR_CUDA(cudaMemcpyAsync(&herr, st.err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    if (herr) return fail(WR_ETIMEDOUT, "tensor-core projection: a bounded wait ran out");
    return WR_OK;
}

wr_status blackbox_apply(wr_ctx *ctx, const wr_matrix *mat, const wr_params &prm, const uint32_t *d_in,
                         uint32_t *d_out, int64_t width) {
    if (width < 1 || width > 32) return fail(WR_EINVAL, "width must be in 1..32");
    wr_params p2 = prm;
    p2.n = (uint32_t)width;
    p2.m = 1;
    Resolved r;
    WR_TRY(resolve(mat, &p2, r));
    SeqState st;
    WR_TRY(seq_setup(ctx, mat, r, st, false));
    cudaStream_t s = ctx->stream;
    if (r.N > 0) {
        k_scale_pad<<<blocks_for(r.N * r.nv, 256), 256, 0, s>>>(r.N, (int)width, r.nv, d_in,
                                                               st.D1.as<uint32_t>(), st.T.as<uint32_t>(), r.nmap,
                                                               st.mp);
        WR_LAUNCHED(ctx);
    }
    WR_TRY(launch_pass(ctx, r.nv, *st.first, st.slabs1, st.T.as<uint32_t>(), st.Wb.as<uint32_t>(),
                       st.D2.as<uint32_t>(), st.acc1.as<unsigned long long>(), st.mp, nullptr, st.wl1));
    // second pass scaled by D1 (not D1^2): out = D1 A^T D2 A D1 in
    WR_TRY(launch_pass(ctx, r.nv, *st.second, st.slabs2, st.Wb.as<uint32_t>(), st.T.as<uint32_t>(),
                       st.D1.as<uint32_t>(), st.acc2.as<unsigned long long>(), st.mp, nullptr, st.wl2));
    if (r.N > 0) {
        k_unpad<<<blocks_for(r.N * width, 256), 256, 0, s>>>(r.N, (int)width, r.nv, st.T.as<uint32_t>(), d_out,
                                                             r.nmap);
        WR_LAUNCHED(ctx);
    }
    WR_CUDA(cudaStreamSynchronize(s));
    return WR_OK;
}

}  // namespace wr

// ---------------------------------------------------------------------------
namespace wr {

// Several jobs on one matrix in one sequence loop (batches: the paper's rank
// over Q takes the same matrix modulo several primes, Section 2.5).  Jobs
// with the same matrix, m = n, side and length (any primes and seeds) each
// carry X beside Y; their slices of 2 nv columns sit side by side in one
// block, so one pair of SpMM passes per application serves them all: the
// exact int64 row sums do not depend on the prime, and the epilogue reduces
// each slice modulo its own prime and scales it by its own diagonal.  The
// Gram projections then run per job on its slice.  Every job's sequence is
// the one it has alone, bit for bit.

bool multi_eligible(const wr_ctx *ctx, const Resolved &r) {
    // at least two jobs of 2 nv columns per block of at most 64, and slices of
    // at least 4 columns (the block is at least 16 columns wide: 4 slices)
    return pairs_generic(ctx, r) && 4 * r.nv <= 64 && r.nv >= 2;
}

int multi_max_jobs(const Resolved &r) { return std::min(MULTI_MAX_JOBS, 64 / (2 * r.nv)); }

wr_status run_sequence_multi(wr_ctx *ctx, const wr_matrix *mat, const std::vector<Resolved> &rs_in,
                             const std::vector<uint32_t *> &d_S, double *seq_ms, const std::vector<SeqFeed *> *feeds) {
    const int G = (int)rs_in.size();
    if (G < 1 || G > MULTI_MAX_JOBS || (int)d_S.size() != G) return fail(WR_EINVAL, "multi-job sequence: 1..4 jobs");
    std::vector<Resolved> rs = rs_in;
    for (auto &r : rs) {
        r.paired = true;
        r.nvs = 2 * r.nv;
    }
    const Resolved &r0 = rs[0];
    for (const auto &r : rs)
        if (r.m != r0.m || r.n != r0.n || r.side != r0.side || r.L != r0.L || !multi_eligible(ctx, r))
            return fail(WR_EINVAL, "multi-job sequence: jobs must share m = n, side and length");
    const int jw = 2 * r0.nv;
    const int W = std::max(16, padded_width(G * jw));
    if (W > 64 || W / jw > MULTI_MAX_JOBS) return fail(WR_EINVAL, "multi-job sequence: block wider than 64 columns");
    int jw_log = 0;
    while ((1 << jw_log) < jw) jw_log++;
    const int64_t N = r0.N, M = r0.M, L = r0.L;
    const int64_t E = (int64_t)r0.m * r0.n;
    cudaStream_t s = ctx->stream;
    cudaEvent_t e1, e2;
    WR_CUDA(cudaEventCreate(&e1));
    WR_CUDA(cudaEventCreateWithFlags(&e2, cudaEventBlockingSync));
    const Sell *first = r0.side == 0 ? &mat->a : &mat->at;
    const Sell *second = r0.side == 0 ? &mat->at : &mat->a;
    int v1 = 0, v2 = 0;
    WR_TRY(lane_width_for(ctx, mat, *first, W, &v1));
    WR_TRY(lane_width_for(ctx, mat, *second, W, &v2));
    DevBuf T, Wb, acc1, acc2, counter, err;
    WR_TRY(dev_alloc(ctx, T, sizeof(uint32_t) * std::max<int64_t>(N * W, 1)));
    WR_TRY(dev_alloc(ctx, Wb, sizeof(uint32_t) * std::max<int64_t>(M * W, 1)));
    WR_TRY(dev_alloc(ctx, acc1, sizeof(unsigned long long) * std::max<int64_t>(first->nsplit * W, 1)));
    WR_TRY(dev_alloc(ctx, acc2, sizeof(unsigned long long) * std::max<int64_t>(second->nsplit * W, 1)));
    WR_TRY(dev_alloc(ctx, counter, sizeof(int)));
    WR_TRY(dev_alloc(ctx, err, sizeof(int)));
    WR_CUDA(cudaMemsetAsync(T.ptr, 0, T.bytes, s));  // slices past the last job stay zero
    WR_CUDA(cudaMemsetAsync(acc1.ptr, 0, acc1.bytes, s));
    WR_CUDA(cudaMemsetAsync(acc2.ptr, 0, acc2.bytes, s));
    WR_CUDA(cudaMemsetAsync(counter.ptr, 0, sizeof(int), s));
    WR_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    struct Job {
        ModP mp;
        DevBuf D1, D2, d1sq, xh, w2, s_raw;
    };
    std::vector<Job> jobs(G);
    MultiEpi me1, me2;
    me1.jobs = me2.jobs = W >> jw_log;
    me1.jw_log = me2.jw_log = jw_log;
    for (int g = 0; g < G; g++) {
        const Resolved &r = rs[g];
        Job &j = jobs[g];
        j.mp = make_modp(r.p);
        WR_TRY(dev_alloc(ctx, j.D1, sizeof(uint32_t) * std::max<int64_t>(N, 1)));
        WR_TRY(dev_alloc(ctx, j.D2, sizeof(uint32_t) * std::max<int64_t>(M, 1)));
        WR_TRY(dev_alloc(ctx, j.d1sq, sizeof(uint32_t) * std::max<int64_t>(N, 1)));
        WR_TRY(dev_alloc(ctx, j.xh, sizeof(uint32_t) * std::max<int64_t>(N, 1)));
        WR_TRY(dev_alloc(ctx, j.w2, sizeof(uint32_t) * std::max<int64_t>(M, 1)));
        WR_TRY(dev_alloc(ctx, j.s_raw, sizeof(unsigned long long) * std::max<int64_t>(L * E, 1)));
        WR_CUDA(cudaMemsetAsync(j.s_raw.ptr, 0, j.s_raw.bytes, s));
        if (N > 0) {
            k_derive_diag<<<blocks_for(N, 256), 256, 0, s>>>(r.seed, TAG_D1, N, r.p, j.D1.as<uint32_t>(), r.nmap);
            WR_LAUNCHED(ctx);
            k_prepare<<<blocks_for(N, 128), 128, 0, s>>>(N, r.m, r.n, r.nv, r.seed, r.xtag, r.xwidth, r.ystride,
                                                         r.ycol0, 0, 1, j.D1.as<uint32_t>(), T.as<uint32_t>() + g * jw,
                                                         j.xh.as<uint32_t>(), j.d1sq.as<uint32_t>(), r.nmap, j.mp, W);
            WR_LAUNCHED(ctx);
        }
        if (M > 0) {
            k_derive_diag<<<blocks_for(M, 256), 256, 0, s>>>(r.seed, TAG_D2, M, r.p, j.D2.as<uint32_t>(), r.mmap);
            WR_LAUNCHED(ctx);
            k_inv_diag<<<blocks_for(M, 256), 256, 0, s>>>(M, j.D2.as<uint32_t>(), j.w2.as<uint32_t>(), j.mp);
            WR_LAUNCHED(ctx);
        }
    }
    for (int g = 0; g < me1.jobs; g++) {
        const Job &j = jobs[g < G ? g : 0];  // slices past the last job: zero columns, any valid modulus
        me1.mp[g] = me2.mp[g] = j.mp;
        me1.scale[g] = j.D2.as<uint32_t>();
        me2.scale[g] = j.d1sq.as<uint32_t>();
    }
    auto grams = [&](bool w_side, int tmul, int toff) -> wr_status {
        for (int g = 0; g < G; g++) {
            Job &j = jobs[g];
            if (w_side)
                WR_TRY(launch_gram_to(ctx, rs[g], j.mp, M, j.w2.as<uint32_t>(), Wb.as<uint32_t>() + g * jw, tmul, toff,
                                      W, r0.nv, j.s_raw.as<unsigned long long>(), counter.as<int>(), err.as<int>()));
            else
                WR_TRY(launch_gram_to(ctx, rs[g], j.mp, N, j.xh.as<uint32_t>(), T.as<uint32_t>() + g * jw, tmul, toff,
                                      W, r0.nv, j.s_raw.as<unsigned long long>(), counter.as<int>(), err.as<int>()));
        }
        return WR_OK;
    };
    if (L > 0) WR_TRY(grams(false, 2, 0));  // S_0
    // fed mode: after every group the terms it finished are reduced into
    // each job's sequence and an event published to that job's sigma-basis
    int64_t published = 0;
    auto publish = [&](int64_t to) -> wr_status {
        for (int g = 0; g < G; g++) {
            if (to > published) {
                k_reduce_seq<<<blocks_for((to - published) * E, 256), 256, 0, s>>>(
                    (to - published) * E, jobs[g].s_raw.as<unsigned long long>() + published * E,
                    d_S[g] + published * E, jobs[g].mp);
                WR_LAUNCHED(ctx);
            }
            SeqFeed *fd = (*feeds)[g];
            cudaEvent_t ev;
            WR_CUDA(cudaEventCreateWithFlags(&ev, WAIT_EVENT_FLAGS));
            cudaError_t ce = cudaEventRecord(ev, s);
            {
                std::lock_guard<std::mutex> lk(fd->mu);
                fd->ev.push_back(ev);  // the feed's owner destroys it
                fd->ready.push_back(ce == cudaSuccess ? to : -1);
            }
            fd->cv.notify_all();
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaEventRecord");
        }
        published = to;
        return WR_OK;
    };
    if (feeds) WR_TRY(publish(std::min<int64_t>(1, L)));
    WR_CUDA(cudaEventRecord(e1, s));
    const SellView f = view(*first), sc = view(*second);
    auto iteration = [&]() -> wr_status {
        WR_TRY(launch_spmm_multi(ctx, W, f, T.as<uint32_t>(), Wb.as<uint32_t>(), acc1.as<unsigned long long>(), me1,
                                 counter.as<int>(), v1));
        WR_TRY(launch_spmm_multi(ctx, W, sc, Wb.as<uint32_t>(), T.as<uint32_t>(), acc2.as<unsigned long long>(), me2,
                                 nullptr, v2));
        WR_TRY(grams(true, 2, -1));
        return grams(false, 2, 0);
    };
    const int64_t terms = std::max<int64_t>(L - 1, 0), iters = (terms + 1) / 2;
    const int64_t Gk = 64;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_launches = 0;
    if (iters >= Gk) {
        const int64_t before = ctx->launches;
        WR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        wr_status cst = WR_OK;
        for (int64_t i = 0; i < Gk && cst == WR_OK; i++) cst = iteration();
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        graph_launches = ctx->launches - before;
        ctx->launches = before;
        if (cst != WR_OK) { if (graph) cudaGraphDestroy(graph); return cst; }
        WR_CUDA(ce);
        ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ce, "cudaGraphInstantiate"); }
    }
    wr_status loop_st = WR_OK;
    int64_t done = 0;
    while (done < iters && loop_st == WR_OK) {
        const int64_t todo = std::min(Gk, iters - done);
        if (todo == Gk && exec) {
            cudaError_t ce = cudaGraphLaunch(exec, s);
            if (ce != cudaSuccess) loop_st = cuda_fail(ce, "cudaGraphLaunch");
            ctx->launches += graph_launches;
        } else {
            for (int64_t i = 0; i < todo && loop_st == WR_OK; i++) loop_st = iteration();
        }
        done += todo;
        if (feeds && loop_st == WR_OK) loop_st = publish(std::min<int64_t>(2 * done + 1, L));
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    WR_TRY(loop_st);
    for (int g = 0; g < G && L * E > 0 && !feeds; g++) {
        k_reduce_seq<<<blocks_for(L * E, 256), 256, 0, s>>>(L * E, jobs[g].s_raw.as<unsigned long long>(), d_S[g],
                                                           jobs[g].mp);
        WR_LAUNCHED(ctx);
    }
    int herr = 0;
    WR_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaEventRecord(e2, s));
    WR_CUDA(cudaEventSynchronize(e2));
    float b = 0;
    cudaEventElapsedTime(&b, e1, e2);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (herr) return fail(WR_ETIMEDOUT, "tensor-core projection: a bounded wait ran out");
    if (seq_ms) *seq_ms = b;
    return WR_OK;
}

}  // namespace wr

// ---------------------------------------------------------------------------
// Black-box application without device allocation.
//
// For callers that must not allocate device memory once they are running:
// code that lives inside another program's fixed device-memory arena (where
// cudaMalloc would fail or fragment the arena), or latency-critical loops that
// cannot afford an allocation (cudaMalloc and cudaFree may synchronise the
// device).  All temporaries of one application (the padded input block, the
// intermediate block, both diagonals and the split-row accumulators) are
// carved out of one fixed array that exists once per device for the life of
// the process.

// 32 MiB of scratch per device, reserved when the library's device code is
// loaded on that device.
static __device__ __align__(256) unsigned char wr_noalloc_scratch[32u << 20];

namespace wr {

constexpr size_t NOALLOC_SCRATCH_BYTES = sizeof(wr_noalloc_scratch);

// Device address of the scratch array, looked up once per device and
// context (the first call on a device does it, with that device current).
// The address belongs to the device's primary context: if the caller resets
// the device (cudaDeviceReset), the context that follows gets a new copy of
// the array, so the lookup is keyed by the context's unique ID (cuCtxGetId,
// through the runtime's driver entry points) and repeated when it changes.
// Where that ID is not available the address is looked up on every call.
static void *g_noalloc_addr[128];
static unsigned long long g_noalloc_ctx[128];
static std::mutex g_noalloc_mu;

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// unique ID of the calling thread's current context, 0 if unknown
static unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    void *c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == 0 && c && get_id(c, &id) == 0) return id;
    return 0;
}

static wr_status noalloc_scratch_address(int device, void **out) {
    if (device < 0 || device >= 128) return fail(WR_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    const unsigned long long id = current_context_id();
    if (!g_noalloc_addr[device] || id == 0 || g_noalloc_ctx[device] != id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, wr_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[device] = p;
        g_noalloc_ctx[device] = current_context_id();  // the context exists now
    }
    *out = g_noalloc_addr[device];
    return WR_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

wr_status blackbox_apply_noalloc(wr_ctx *ctx, const wr_matrix *mat, const wr_params &prm,
                                 const uint32_t *d_in, uint32_t *d_out, int64_t width) {
    if (width < 1 || width > 32) return fail(WR_EINVAL, "width must be in 1..32");
    wr_params p2 = prm;
    p2.n = (uint32_t)width;
    p2.m = 1;
    Resolved r;
    WR_TRY(resolve(mat, &p2, r));
    const Sell *first = r.side == 0 ? &mat->a : &mat->at;
    const Sell *second = r.side == 0 ? &mat->at : &mat->a;
    const int nv = r.nv;
    // layout of the scratch array
    const size_t oT = 0;
    const size_t oW = oT + align256(sizeof(uint32_t) * (size_t)r.N * nv);
    const size_t oD1 = oW + align256(sizeof(uint32_t) * (size_t)r.M * nv);
    const size_t oD2 = oD1 + align256(sizeof(uint32_t) * (size_t)r.N);
    const size_t oA1 = oD2 + align256(sizeof(uint32_t) * (size_t)r.M);
    const size_t nA1 = sizeof(unsigned long long) * (size_t)first->nsplit * nv;
    const size_t oA2 = oA1 + align256(nA1);
    const size_t nA2 = sizeof(unsigned long long) * (size_t)second->nsplit * nv;
    const size_t need = oA2 + align256(nA2);
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(WR_EINVAL, "this matrix and width need " + std::to_string(need) +
                                   " bytes of scratch; the allocation-free call has " +
                                   std::to_string(NOALLOC_SCRATCH_BYTES) + " bytes (use wr_blackbox_apply_device)");
    void *base = nullptr;
    WR_TRY(noalloc_scratch_address(ctx->device, &base));
    unsigned char *b = static_cast<unsigned char *>(base);
    uint32_t *T = reinterpret_cast<uint32_t *>(b + oT);
    uint32_t *Wb = reinterpret_cast<uint32_t *>(b + oW);
    uint32_t *D1 = reinterpret_cast<uint32_t *>(b + oD1);
    uint32_t *D2 = reinterpret_cast<uint32_t *>(b + oD2);
    unsigned long long *acc1 = reinterpret_cast<unsigned long long *>(b + oA1);
    unsigned long long *acc2 = reinterpret_cast<unsigned long long *>(b + oA2);
    const ModP mp = make_modp(r.p);
    cudaStream_t s = ctx->stream;
    // the split-row accumulators must start at zero; the scratch keeps
    // whatever the previous call left there
    if (nA1) WR_CUDA(cudaMemsetAsync(acc1, 0, nA1, s));
    if (nA2) WR_CUDA(cudaMemsetAsync(acc2, 0, nA2, s));
    if (r.N > 0) {
        k_derive_diag<<<blocks_for(r.N, 256), 256, 0, s>>>(r.seed, TAG_D1, r.N, r.p, D1, r.nmap);
        WR_LAUNCHED(ctx);
    }
    if (r.M > 0) {
        k_derive_diag<<<blocks_for(r.M, 256), 256, 0, s>>>(r.seed, TAG_D2, r.M, r.p, D2, r.mmap);
        WR_LAUNCHED(ctx);
    }
    if (r.N > 0) {
        k_scale_pad<<<blocks_for(r.N * nv, 256), 256, 0, s>>>(r.N, (int)width, nv, d_in, D1, T, r.nmap, mp);
        WR_LAUNCHED(ctx);
    }
    WR_TRY(launch_spmm(ctx, nv, view(*first), T, Wb, D2, acc1, mp, nullptr));
    WR_TRY(launch_spmm(ctx, nv, view(*second), Wb, T, D1, acc2, mp, nullptr));
    if (r.N > 0) {
        k_unpad<<<blocks_for(r.N * width, 256), 256, 0, s>>>(r.N, (int)width, nv, T, d_out, r.nmap);
        WR_LAUNCHED(ctx);
    }
    WR_CUDA(cudaStreamSynchronize(s));
    return WR_OK;
}

}  // namespace wr
