// The projection's weighted Gram products on the tensor cores.
//
// Two terms per application of A~ (Section 2.3: A~ = D1 A^T D2 A D1 is
// symmetric; Table tab:r-opp col. 3 is the paper's dot-product step) come from
// products of the form
//
//   G = sum_r w_r L_r^T R_r  mod p,   L_r = t[r][0 .. m),  R_r = t[r][yoff .. yoff + n)
//
// over the N rows of a block t (the symmetric projection: L = R; X beside Y:
// the X and Y halves of the paired block).  They are computed exactly from
// half-precision products of 8-bit digits.  A residue x < 2^31 is written in
// balanced digits x = sum_i d_i 2^{8i}: with y = x + 0x808080, d_i = byte_i(y) -
// 128 for i < 3 and d_3 = byte_3(y) in [0, 128].  Every digit is an integer of
// magnitude <= 128 (exact in fp16), a digit product is at most 2^14, so the
// fp32 sums of GT_DRAIN * 64 = 512 rows stay below 2^23 and are exact.
//
// Per tile of 64 rows (the MMA's K), one tcgen05 MMA chain computes
//   D[i*32 + a][j*NB + b] = sum_r d_i(w_r L_r[a]) d_j(R_r[b])
// (kind::f16 with fp16 operands, M = 128 = 4 digits x 32 left columns, N = 4
// digits x NB right columns, fp32 in tensor memory); every 512 rows the eight
// converter warps drain the accumulator (TMEM lane: digit i = warp % 4, column
// a = lane; half warp / 4 of the right columns) into exact int64 sums
// acc[b] += sum_j 2^{8j} D[i*32 + a][j*NB + b], and at the end
//   G[a][b] = sum_i 2^{8i} acc_i[a][b]  mod p.
// The rows of t and their weights reach shared memory by 1-D bulk copies
// (up to five tiles in flight per block, two blocks per SM), eight warps
// rewrite them as digit tiles in the MMA's swizzled layout, and a ninth warp
// issues the MMAs, commits them to an mbarrier and requests the next rows, so
// that issuing never holds up the conversion; operand tiles are
// double-buffered.  Every wait is bounded: after WAIT_NS the block records an
// error, waits (bounded) for its copies and MMAs in flight, frees its tensor
// memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "wr_internal.cuh"
#include "wr_tc.cuh"

namespace wr {

namespace {

constexpr int GT_CONV = 256;              // converter threads (warps 0-7)
constexpr int GT_THREADS = GT_CONV + 32;  // and the issuer warp
constexpr int GT_KT = 64;     // rows per tile
constexpr int GT_DRAIN = 8;   // tiles per drain of the accumulator (512 rows)
constexpr uint64_t GT_WAIT_NS = 2000000000ull;
constexpr int GT_ERR_TIMEOUT = 1;

template <int NB, int RB>
struct GramShape {
    static constexpr int TN = 4 * NB;                      // B rows (N of the MMA)
    static constexpr uint32_t ABYTES = 128u * 128u;        // A tile: 128 rows x 128 bytes
    static constexpr uint32_t BBYTES = (uint32_t)TN * 128u;
    static constexpr uint32_t OPB = ABYTES + BBYTES;       // one operand stage
    static constexpr uint32_t RAWB = (uint32_t)GT_KT * RB; // one raw tile
    static constexpr uint32_t TMEM_COLS = TN < 32 ? 32 : TN;
    static constexpr uint32_t WB = (uint32_t)GT_KT * 4;   // one tile's weights
    // raw tiles in flight per block (two blocks a SM): five for rows of up to
    // 128 bytes (32 KB in flight a block, what the shared memory of two
    // blocks allows), two for the wider rows
    static constexpr int NS = RB <= 128 ? 5 : 2;
    static constexpr size_t SMEM = 1024 + 2 * (size_t)OPB + NS * ((size_t)RAWB + WB) + 128;
    static_assert(NB == 8 || NB == 16 || NB == 32, "NB");
    static_assert(RB % 16 == 0 && RB >= 32 && RB <= 256, "RB");
    static_assert(4u * 32u * NB * 4u <= NS * RAWB, "reduction area");
    static_assert(2 * (SMEM + 1024) <= 228 * 1024, "two blocks a SM");
};

// Digit I of two consecutive values (y = x + 0x808080 each) as an fp16 pair:
// the two bytes are placed under 0x64 (fp16 bits 0x64ee = 1024 + e, exact for
// e < 1024) and 1024 + 128 (digits 0..2) or 1024 (digit 3) is subtracted in
// one packed half-precision subtraction; every result is an integer of
// magnitude <= 128, exact.  The lower K index goes to the lower half.
template <int I>
__device__ __forceinline__ uint32_t digit_h2(uint32_t y0, uint32_t y1) {
    const uint32_t t = __byte_perm(y0, y1, I | ((I + 4) << 4));  // [b_I(y0), b_I(y1), ., .]
    const uint32_t h = __byte_perm(t, 0x64646464u, 0x4140);      // [b_I(y0), 0x64, b_I(y1), 0x64]
    uint32_t r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(h), "r"(I < 3 ? 0x64806480u : 0x64006400u));
    return r;
}

// byte offsets in a swizzled tile of the 16-byte chunk c of the 4 digit rows
// row0 + i * stride (the same for every tile a thread converts)
__device__ __forceinline__ void digit_offsets(int row0, int stride, int c, uint32_t (&off)[4]) {
#pragma unroll
    for (int i = 0; i < 4; i++) off[i] = tc::sw128_chunk((uint32_t)(row0 + i * stride), (uint32_t)c);
}

// the 4 digit rows of 8 consecutive K values into their chunks (off)
__device__ __forceinline__ void put_digits(unsigned char *tile, const uint32_t (&off)[4], const uint32_t (&x)[8]) {
    uint32_t y[8];
#pragma unroll
    for (int u = 0; u < 8; u++) y[u] = x[u] + 0x808080u;
#define WR_DIGIT_ROW(I)                                                                              \
    {                                                                                                \
        uint4 q;                                                                                     \
        q.x = digit_h2<I>(y[0], y[1]);                                                               \
        q.y = digit_h2<I>(y[2], y[3]);                                                               \
        q.z = digit_h2<I>(y[4], y[5]);                                                               \
        q.w = digit_h2<I>(y[6], y[7]);                                                               \
        *reinterpret_cast<uint4 *>(tile + off[I]) = q;                                               \
    }
    WR_DIGIT_ROW(0)
    WR_DIGIT_ROW(1)
    WR_DIGIT_ROW(2)
    WR_DIGIT_ROW(3)
#undef WR_DIGIT_ROW
}

// G into s_raw[k] (k = tmul * counter + toff; skipped unless 0 <= k < L): the
// per-block result reduced mod p, then added with exact uint64 atomics.
// w: the N weights in Montgomery form (mont_mul(w_r, x) = w_r x mod p); t and w
// 16-byte aligned (bulk copies).
//
// Roles: warps 0-7 convert (tile tl: wait for its raw rows and for the MMAs
// that last read its operand stage, write the digit tiles, one arrival per
// warp on conv[stage]); warp 8's first lane issues (wait on conv[stage],
// the four MMAs of the tile, the commit to mma[stage], the bulk copies of the
// tile GT_NS ahead into the raw stage just converted), so that the issue
// never holds up a converter.  Every GT_DRAIN tiles the converters drain the
// accumulator (warp w: digit row w % 4 of the left factor, half w / 4 of the
// right factor's columns) and arrive on drained, which the issuer waits for
// before the next group overwrites the accumulator.  All waits are bounded
// mbarrier waits; a wait that runs out sets a shared flag that every role
// polls, and the issuer then lets the copies and MMAs in flight finish.
template <int NB, int RB>
__global__ void __launch_bounds__(GT_THREADS, 2)
    k_gram_tc(int64_t N, int m, int n, const uint32_t *__restrict__ w, const uint32_t *__restrict__ t, int yoff,
              unsigned long long *__restrict__ s_raw, const int *__restrict__ term_counter, int tmul, int toff,
              int64_t L, ModP mp, int *__restrict__ err) {
    using S = GramShape<NB, RB>;
    constexpr int RW = RB / 4;      // residues per raw row
    constexpr int HB = NB / 2;      // right-factor columns a draining thread holds
    constexpr uint32_t IDESC = tc::idesc_f16_f32(128, S::TN);
    const int64_t k_term = term_counter ? (int64_t)tmul * *term_counter + toff : (int64_t)toff;
    if (k_term < 0 || k_term >= L) return;  // the same for every block

    extern __shared__ unsigned char gsm[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(gsm) + 1023) & ~uintptr_t(1023));
    unsigned char *raw = base + 2 * S::OPB;
    uint32_t *wts = reinterpret_cast<uint32_t *>(raw + S::NS * S::RAWB);  // NS x 64 weights
    uint64_t *bar_raw = reinterpret_cast<uint64_t *>(wts + S::NS * GT_KT);
    uint64_t *bar_mma = bar_raw + S::NS;   // [2] MMAs of an operand stage done
    uint64_t *bar_conv = bar_mma + 2;      // [2] operand stage converted
    uint64_t *bar_drain = bar_conv + 2;    // accumulator drained
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar_drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == GT_CONV / 32;
    const int64_t tiles = (N + GT_KT - 1) / GT_KT;
    const int64_t t_begin = tiles * blockIdx.x / gridDim.x;
    const int64_t ntile = tiles * (blockIdx.x + 1) / gridDim.x - t_begin;

    // both operand stages start at zero: digit rows of absent columns stay zero
    for (uint32_t i = (uint32_t)tid * 16u; i < 2u * S::OPB; i += GT_THREADS * 16u)
        *reinterpret_cast<uint4 *>(base + i) = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int s = 0; s < S::NS; s++) tc::mbar_init(&bar_raw[s], 1);
        tc::mbar_init(&bar_mma[0], 1);
        tc::mbar_init(&bar_mma[1], 1);
        tc::mbar_init(&bar_conv[0], GT_CONV / 32);
        tc::mbar_init(&bar_conv[1], GT_CONV / 32);
        tc::mbar_init(bar_drain, GT_CONV / 32);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, S::TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int64_t issued = 0, committed = 0;  // (issuer) raw tiles requested, MMA commits
    auto issue = [&](int64_t tl) {
        const int s = (int)(tl % S::NS);
        const int64_t r0 = (t_begin + tl) * GT_KT;
        const uint32_t rows = (uint32_t)min64(GT_KT, N - r0);
        const uint32_t wrows = rows & ~3u;  // whole 16-byte groups of weights; the rest by plain loads
        tc::mbar_arrive_expect_tx(&bar_raw[s], rows * (uint32_t)RB + wrows * 4u);
        tc::bulk_g2s(raw + s * S::RAWB, t + r0 * RW, rows * (uint32_t)RB, &bar_raw[s]);
        if (wrows) tc::bulk_g2s(wts + s * GT_KT, w + r0, wrows * 4u, &bar_raw[s]);
    };

    long long acc[HB];
#pragma unroll
    for (int b = 0; b < HB; b++) acc[b] = 0;

    if (issuer) {
        if (lane == 0) {
            for (; issued < ntile && issued < S::NS; issued++) issue(issued);
            for (int64_t tl = 0; tl < ntile; tl++) {
                const int so = (int)(tl & 1), g = (int)(tl % GT_DRAIN);
                if (*abort_flag) break;
                bool ok = tc::mbar_wait(&bar_conv[so], (uint32_t)((tl >> 1) & 1), GT_WAIT_NS);
                // a new group overwrites the accumulator: the last one's drain must be done
                if (ok && g == 0 && tl > 0)
                    ok = tc::mbar_wait(bar_drain, (uint32_t)(((tl / GT_DRAIN) - 1) & 1), GT_WAIT_NS);
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                tc::tc_fence_after();
                unsigned char *opA = base + so * S::OPB, *opB = opA + S::ABYTES;
                const uint32_t a0 = tc::smem_addr(opA), b0 = tc::smem_addr(opB);
#pragma unroll
                for (int ks = 0; ks < GT_KT / 16; ks++)
                    tc::mma_f16(tmem, tc::sdesc_k_sw128(a0 + 32u * ks), tc::sdesc_k_sw128(b0 + 32u * ks), IDESC,
                                 (ks > 0 || g > 0) ? 1u : 0u);
                tc::mma_commit(&bar_mma[so]);
                committed++;
                // the raw stage of this tile has been converted: refill it
                if (issued < ntile) {
                    tc::fence_proxy_async_smem();
                    issue(issued);
                    issued++;
                }
            }
        }
        __syncwarp();
    } else {
        // this thread's chunks: left factor chunk c = warp (rows 8c .. 8c + 7),
        // column a = lane; right factor chunk tid / NB, column tid % NB
        const int ca = warp, a = lane, cb = tid / NB, b = tid % NB;
        const bool do_l = a < m, do_r = tid < 8 * NB && b < n;
        uint32_t offL[4], offR[4];
        digit_offsets(a, 32, ca, offL);
        digit_offsets(b, NB, cb & 7, offR);
        for (int64_t tl = 0; tl < ntile; tl++) {
            const int sr = (int)(tl % S::NS), so = (int)(tl & 1);
            const int g = (int)(tl % GT_DRAIN);
            if (*abort_flag) break;
            unsigned char *opA = base + so * S::OPB, *opB = opA + S::ABYTES;
            // the raw rows have landed; the operand stage's previous MMAs are done
            bool ok = tc::mbar_wait(&bar_raw[sr], (uint32_t)((tl / S::NS) & 1), GT_WAIT_NS);
            if (ok && tl >= 2) ok = tc::mbar_wait(&bar_mma[so], (uint32_t)(((tl >> 1) - 1) & 1), GT_WAIT_NS);
            if (!ok) {
                *abort_flag = 1;
                break;
            }
            const int64_t r0 = (t_begin + tl) * GT_KT;
            const int rows = (int)min64(GT_KT, N - r0);
            const uint32_t *rw = reinterpret_cast<const uint32_t *>(raw + sr * S::RAWB);
            const uint32_t *ws = wts + sr * GT_KT;
            const int wrows = rows & ~3;
            if (rows == GT_KT) {
                // a whole tile: every row and weight is in shared memory
                if (do_l) {
                    uint32_t x[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) x[u] = mont_mul(ws[8 * ca + u], rw[(8 * ca + u) * RW + a], mp);
                    put_digits(opA, offL, x);
                }
                if (do_r) {
                    uint32_t x[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) x[u] = rw[(8 * cb + u) * RW + yoff + b];
                    put_digits(opB, offR, x);
                }
            } else {
                if (do_l) {
                    // left factor, weighted (the last weights past a 16-byte group by plain loads)
                    uint32_t x[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int rr = 8 * ca + u;
                        const uint32_t wv = rr < wrows ? ws[rr] : (rr < rows ? __ldg(w + r0 + rr) : 0u);
                        x[u] = rr < rows ? mont_mul(wv, rw[rr * RW + a], mp) : 0u;
                    }
                    put_digits(opA, offL, x);
                }
                if (do_r) {
                    uint32_t x[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int rr = 8 * cb + u;
                        x[u] = rr < rows ? rw[rr * RW + yoff + b] : 0u;
                    }
                    put_digits(opB, offR, x);
                }
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bar_conv[so]);
            if (g == GT_DRAIN - 1 || tl == ntile - 1) {
                // drain: the accumulator of this group into the int64 sums
                // (the commit of this tile covers every earlier MMA)
                if (!tc::mbar_wait(&bar_mma[so], (uint32_t)((tl >> 1) & 1), GT_WAIT_NS)) {
                    *abort_flag = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
                const int hf = warp >> 2;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    uint32_t v[HB];
                    tc::tmem_ldn<HB>(tmem + lanes + (uint32_t)(j * NB + hf * HB), v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int b = 0; b < HB; b++) acc[b] += (long long)__float2int_rn(__uint_as_float(v[b])) << (8 * j);
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(bar_drain);
            }
        }
    }

    __syncthreads();
    const bool aborted = *abort_flag != 0;
    if (aborted) {
        // record the error, let the copies and MMAs in flight finish (bounded)
        if (issuer && lane == 0) {
            atomicExch(err, GT_ERR_TIMEOUT);
            for (int64_t tl = max64(0, issued - S::NS); tl < issued; tl++)
                tc::mbar_wait(&bar_raw[tl % S::NS], (uint32_t)((tl / S::NS) & 1), GT_WAIT_NS);
            if (committed > 0) {
                const int64_t last = committed - 1;
                tc::mbar_wait(&bar_mma[last & 1], (uint32_t)((last >> 1) & 1), GT_WAIT_NS);
            }
        }
        tc::tc_fence_before();
        __syncthreads();
    } else {
        // G[a][b] = sum_i 2^{8i} acc_i[a][b] mod p: per digit row reduced and
        // scaled by the converters, summed over the digits below
        uint32_t *red = reinterpret_cast<uint32_t *>(raw);
        if (!issuer) {
            const int i = warp & 3, hf = warp >> 2;
            const uint32_t sc = powm(256u % mp.p, (uint32_t)i, mp);  // 2^{8 i} mod p
#pragma unroll
            for (int b = 0; b < HB; b++) red[(i * 32 + lane) * NB + hf * HB + b] = mulm(red_s64(acc[b], mp), sc, mp);
        }
        __syncthreads();
        unsigned long long *dst = s_raw + (size_t)k_term * m * n;
        for (int e = tid; e < m * n; e += GT_THREADS) {
            const int a = e / n, b = e % n;
            unsigned long long v = 0;
#pragma unroll
            for (int i = 0; i < 4; i++) v += red[(i * 32 + a) * NB + b];
            const uint32_t r = red64(v, mp);
            if (r) atomicAdd(dst + e, (unsigned long long)r);
        }
        tc::tc_fence_before();
        __syncthreads();
    }
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, S::TMEM_COLS);
    }
}

template <int NB, int RB>
wr_status launch_gram_tc_t(wr_ctx *ctx, int64_t N, int m, int n, const uint32_t *w, const uint32_t *t, int yoff,
                           unsigned long long *s_raw, const int *term_counter, int tmul, int toff, int64_t L,
                           const ModP &mp, int *err) {
    using S = GramShape<NB, RB>;
    static std::once_flag once[8];
    static cudaError_t attr_err[8];
    const int dev = ctx->device & 7;
    std::call_once(once[dev], [&] {
        attr_err[dev] = cudaFuncSetAttribute(k_gram_tc<NB, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)S::SMEM);
    });
    WR_CUDA(attr_err[dev]);
    const int64_t tiles = (N + GT_KT - 1) / GT_KT;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, 2 * (int64_t)ctx->num_sms);  // two blocks a SM
    if (grid == 0) return WR_OK;
    k_gram_tc<NB, RB><<<grid, GT_THREADS, S::SMEM, ctx->stream>>>(N, m, n, w, t, yoff, s_raw, term_counter, tmul,
                                                                  toff, L, mp, err);
    WR_LAUNCHED(ctx);
    return WR_OK;
}

// ------------------------------------------------------------------ tensor-core rate and layout probe
//
// Every block fills a 128 x 64 A tile and a PN x 64 B tile (bf16, the same
// swizzled layout) with small integers, then one thread issues iters chains
// of 4 MMAs (M = 128, N = PN, K = 64) into one accumulator and commits.  With
// out != nullptr block 0 writes D (128 x PN fp32) after its MMAs: the layout
// check compares it with the integer product of the same tiles.
constexpr int PN = 256;

__device__ __forceinline__ int probe_a(int r, int k) { return ((r * 7 + k * 3) % 17) - 8; }
__device__ __forceinline__ int probe_b(int r, int k) { return ((r * 5 + k * 11) % 13) - 6; }

__global__ void __launch_bounds__(128, 1) k_probe_mma(int64_t iters, float *__restrict__ out, int *__restrict__ err) {
    extern __shared__ unsigned char psm[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(psm) + 1023) & ~uintptr_t(1023));
    unsigned char *A = base, *B = base + 128 * 128;
    uint64_t *bar = reinterpret_cast<uint64_t *>(B + PN * 128);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int e = tid; e < 128 * 64; e += 128) {
        const int r = e / 64, k = e % 64;
        *reinterpret_cast<unsigned short *>(A + tc::sw128_chunk(r, k / 8) + (k % 8) * 2) =
            (unsigned short)(__float_as_uint((float)probe_a(r, k)) >> 16);
    }
    for (int e = tid; e < PN * 64; e += 128) {
        const int r = e / 64, k = e % 64;
        *reinterpret_cast<unsigned short *>(B + tc::sw128_chunk(r, k / 8) + (k % 8) * 2) =
            (unsigned short)(__float_as_uint((float)probe_b(r, k)) >> 16);
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, PN);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *slot;
    constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, PN);
    if (tid == 0) {
        const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
        for (int64_t it = 0; it < iters; it++)
#pragma unroll
            for (int ks = 0; ks < 4; ks++)
                tc::mma_f16(tmem, tc::sdesc_k_sw128(a0 + 32u * ks), tc::sdesc_k_sw128(b0 + 32u * ks), IDESC,
                             (it > 0 || ks > 0) ? 1u : 0u);
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, 0, GT_WAIT_NS);
    if (!ok && tid == 0) atomicExch(err, GT_ERR_TIMEOUT);
    tc::tc_fence_after();
    if (ok && out && blockIdx.x == 0) {
        for (int ch = 0; ch < PN / 32; ch++) {
            uint32_t v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32), v);
            tc::tmem_ld_wait();
            for (int cc = 0; cc < 32; cc++) out[(size_t)(warp * 32 + (tid & 31)) * PN + ch * 32 + cc] = __uint_as_float(v[cc]);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, PN);
    }
}

}  // namespace

bool gram_tc_supported(int m, int n, int tstride, int yoff) {
    if (m < 1 || m > 32 || n < 1 || n > 32) return false;
    const int rb = 4 * tstride;
    if (rb != 32 && rb != 64 && rb != 128 && rb != 256) return false;
    const int nb = n <= 8 ? 8 : (n <= 16 ? 16 : 32);
    if (m > tstride || yoff + n > tstride) return false;
    if (nb == 8 && rb > 64) return false;
    if (nb == 16 && (rb < 64 || rb > 128)) return false;
    if (nb == 32 && rb < 128) return false;
    return true;
}

wr_status launch_gram_tc(wr_ctx *ctx, int64_t N, int m, int n, const uint32_t *w, const uint32_t *t, int tstride,
                         int yoff, unsigned long long *s_raw, const int *term_counter, int tmul, int toff, int64_t L,
                         const ModP &mp, int *err) {
    if (!gram_tc_supported(m, n, tstride, yoff)) return fail(WR_EINVAL, "tensor-core Gram: unsupported shape");
    if (N <= 0) return WR_OK;
    const int rb = 4 * tstride;
    const int nb = n <= 8 ? 8 : (n <= 16 ? 16 : 32);
#define WR_GT(NBV, RBV)                                                                                        \
    if (nb == NBV && rb == RBV)                                                                                \
        return launch_gram_tc_t<NBV, RBV>(ctx, N, m, n, w, t, yoff, s_raw, term_counter, tmul, toff, L, mp, err);
    WR_GT(8, 32)
    WR_GT(8, 64)
    WR_GT(16, 64)
    WR_GT(16, 128)
    WR_GT(32, 128)
    WR_GT(32, 256)
#undef WR_GT
    return fail(WR_EINVAL, "tensor-core Gram: unsupported shape");
}

wr_status probe_mma(wr_ctx *ctx, int64_t iters, int blocks, float *d_out, double *ms) {
    // (more shared memory than the tiles need: one block per SM)
    const size_t smem = std::max<size_t>(1024 + 128 * 128 + PN * 128 + 64, 120 * 1024);
    WR_CUDA(cudaFuncSetAttribute(k_probe_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DevBuf err;
    WR_TRY(dev_alloc(ctx, err, sizeof(int)));
    WR_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), ctx->stream));
    cudaEvent_t e0, e1;
    WR_CUDA(cudaEventCreate(&e0));
    WR_CUDA(cudaEventCreate(&e1));
    WR_CUDA(cudaEventRecord(e0, ctx->stream));
    k_probe_mma<<<blocks, 128, smem, ctx->stream>>>(iters, d_out, err.as<int>());
    WR_LAUNCHED(ctx);
    WR_CUDA(cudaEventRecord(e1, ctx->stream));
    WR_CUDA(cudaEventSynchronize(e1));
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int h = 0;
    WR_CUDA(cudaMemcpy(&h, err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) return fail(WR_ETIMEDOUT, "tensor-core probe: an MMA wait ran out");
    return WR_OK;
}

}  // namespace wr
