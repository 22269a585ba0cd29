// Products of polynomial matrices mod p by number-theoretic transforms, for
// the PM-Basis sigma-basis (Section 2.4: "PM-Basis ... reduces this
// computation to polynomial matrix multiplication", FFT primes c 2^k + 1, and
// CRT with several FFT primes when the field itself has no large 2^k-th roots
// of unity, with prod p_i > d n p^2).
//
// C = A B with A (r x s) and B (s x t) polynomial matrices whose entries are
// residues mod p, stored coefficient-major ([coef][row][col]).  Each product
// entry is computed exactly as an integer -- a sum of at most
// s * min(deg A, deg B) + s products below p^2 < 2^62, so below 2^88 for
// s <= 64 and degrees below 2^20 -- from its residues modulo three FFT primes
// whose product exceeds 2^89, and then reduced mod p.  Only the coefficients
// [lo, hi) of C are produced; a cyclic transform of length Lz >= hi whose
// wrapped-around part (coefficients at and above Lz folded onto 0..) stays
// below lo gives exactly those (a middle product when lo > 0).
//
// Transforms: forward decimation in frequency (natural order in, bit-reversed
// out), pointwise products in that order, inverse decimation in time
// (bit-reversed in, natural out); residues in Montgomery form; the stages
// are grouped into passes through shared memory (two passes up to 2^17 points,
// three up to 2^23), each one launch over all polynomials of the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "wr_internal.cuh"

namespace wr {

namespace {

constexpr int NTT_NPRIMES = 3;
constexpr uint32_t NTT_PRIMES[NTT_NPRIMES] = {998244353u, 469762049u, 2013265921u};  // 119 2^23+1, 7 2^26+1, 15 2^27+1
constexpr int NTT_MAX_LOG = 23;  // 2^23 divides every p_i - 1

uint64_t hpow(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = (unsigned __int128)r * a % m;
        a = (unsigned __int128)a * a % m;
        e >>= 1;
    }
    return r;
}

// smallest generator of the multiplicative group mod prime P (checked
// against every prime factor of P - 1)
uint32_t primitive_root(uint32_t P) {
    std::vector<uint64_t> f;
    uint64_t x = P - 1;
    for (uint64_t d = 2; d * d <= x; d++)
        if (x % d == 0) {
            f.push_back(d);
            while (x % d == 0) x /= d;
        }
    if (x > 1) f.push_back(x);
    for (uint32_t g = 2;; g++) {
        bool ok = true;
        for (uint64_t q : f)
            if (hpow(g, (P - 1) / q, P) == 1) { ok = false; break; }
        if (ok) return g;
    }
}

// a (mod p, any p < 2^31) -> Montgomery form mod P, transposed to one
// contiguous run of Lz coefficients per polynomial (zero padded).  Tiles of
// 32 coefficients x 32 entries go through shared memory, so that both the
// reads (along the entries of a coefficient) and the writes (along the
// coefficients of an entry) are coalesced.
constexpr int TR_TILE = 32, TR_ROWS = 8;  // tile edge; thread rows of a 32 x 8 block

__global__ void __launch_bounds__(TR_TILE * TR_ROWS)
    k_ntt_load(const uint32_t *__restrict__ src, int64_t ncoef, int nent, int64_t Lz, uint32_t *__restrict__ dst,
               ModP mP) {
    __shared__ uint32_t tile[TR_TILE][TR_TILE + 1];
    const int tx = threadIdx.x & (TR_TILE - 1), ty = threadIdx.x / TR_TILE;
    const int64_t ktiles = (Lz + TR_TILE - 1) / TR_TILE, etiles = (nent + TR_TILE - 1) / TR_TILE;
    for (int64_t tl = blockIdx.x; tl < ktiles * etiles; tl += gridDim.x) {
        const int64_t k0 = (tl % ktiles) * TR_TILE;
        const int e0 = (int)(tl / ktiles) * TR_TILE;
        __syncthreads();
        if (k0 < ncoef) {
            for (int y = ty; y < TR_TILE; y += TR_ROWS) {
                const int64_t k = k0 + y;
                const int e = e0 + tx;
                tile[y][tx] = (k < ncoef && e < nent) ? to_mont(src[(size_t)k * nent + e] % mP.p, mP) : 0u;
            }
        }
        __syncthreads();
        for (int y = ty; y < TR_TILE; y += TR_ROWS) {
            const int e = e0 + y;
            const int64_t k = k0 + tx;
            if (e < nent && k < Lz) dst[(size_t)e * Lz + k] = k0 < ncoef ? tile[tx][y] : 0u;
        }
    }
}

// tw[j] = w^j (Montgomery form, w_m = w R mod P) for j < count, by square
// and multiply
__global__ void k_twiddles(uint32_t w_m, int64_t count, uint32_t *__restrict__ tw, ModP mP) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x) {
        uint32_t r = mP.r1, b = w_m;
        for (int64_t e = j; e; e >>= 1) {
            if (e & 1) r = mont_mul(r, b, mP);
            b = mont_mul(b, b, mP);
        }
        tw[j] = r;
    }
}

// Several butterfly stages in one pass through shared memory.  The stages
// with half = 2^h for h in [b0, b1) pair elements that differ in one of the
// index bits b0 .. b1 - 1 only, so with e = top 2^b1 + mid 2^b0 + low, a tile
// of all 2^(b1-b0) mid values x 2^LB consecutive low values (LB = min(b0, 5))
// of one (polynomial, top, low block) goes through all of them in shared
// memory: one read and one write of the data per pass instead of per stage.
// DIF (forward): h from b1 - 1 down to b0, (u, v) -> (u + v, (u - v) w^j);
// DIT (inverse): h from b0 up to b1 - 1, (u, v w^j) -> (u + v w^j, u - v w^j);
// j = e mod 2^h, w the 2^(h+1)-th root of unity: w^j = tw[j 2^(lg-1-h+tshift)]
// in a table of the powers of a 2^(lg+tshift)-th root (Montgomery form).
constexpr int NTT_PASS_THREADS = 256;
constexpr int NTT_TILE_LOG = 12;  // 4096 residues (16 KB) per tile

template <bool DIF>
__global__ void __launch_bounds__(NTT_PASS_THREADS)
    k_ntt_pass(uint32_t *__restrict__ a, int64_t npoly, int lg, int b0, int b1, const uint32_t *__restrict__ tw,
               int tshift, ModP mP) {
    __shared__ uint32_t sm[1 << NTT_TILE_LOG];
    const int MB = b1 - b0, LB = b0 < 5 ? b0 : 5;
    const int nlow = 1 << LB, tile = 1 << (MB + LB), half_tile = tile >> 1;
    const int64_t Lz = (int64_t)1 << lg;
    const int lowblocks_log = b0 - LB;
    const int64_t tiles_per_poly = Lz >> (MB + LB);
    for (int64_t tid_tile = blockIdx.x; tid_tile < npoly * tiles_per_poly; tid_tile += gridDim.x) {
        const int64_t poly = tid_tile / tiles_per_poly, rem = tid_tile - poly * tiles_per_poly;
        const int64_t lowblock = rem & (((int64_t)1 << lowblocks_log) - 1), top = rem >> lowblocks_log;
        uint32_t *g = a + poly * Lz + (top << b1) + (lowblock << LB);
        const int64_t lowbase = lowblock << LB;  // low part of e for l = 0
        __syncthreads();
        for (int x = threadIdx.x; x < tile; x += NTT_PASS_THREADS)
            sm[x] = g[((int64_t)(x >> LB) << b0) + (x & (nlow - 1))];
        __syncthreads();
        for (int k = 0; k < MB; k++) {
            const int h = DIF ? b1 - 1 - k : b0 + k;
            const int hh = h - b0, hm = 1 << hh;
            const int sh = lg - 1 - h + tshift;
            for (int y = threadIdx.x; y < half_tile; y += NTT_PASS_THREADS) {
                const int l = y & (nlow - 1), r = y >> LB;
                const int jm = r & (hm - 1), mid0 = ((r >> hh) << (hh + 1)) + jm;
                const int i0 = (mid0 << LB) + l, i1 = i0 + (hm << LB);
                const int64_t j = ((int64_t)jm << b0) + lowbase + l;  // e mod 2^h
                const uint32_t w = tw[j << sh];
                const uint32_t u = sm[i0];
                if (DIF) {
                    const uint32_t v = sm[i1];
                    sm[i0] = addm(u, v, mP);
                    sm[i1] = mont_mul(subm(u, v, mP), w, mP);
                } else {
                    const uint32_t v = mont_mul(sm[i1], w, mP);
                    sm[i0] = addm(u, v, mP);
                    sm[i1] = subm(u, v, mP);
                }
            }
            __syncthreads();
        }
        for (int x = threadIdx.x; x < tile; x += NTT_PASS_THREADS)
            g[((int64_t)(x >> LB) << b0) + (x & (nlow - 1))] = sm[x];
    }
}

// Bit ranges [b0, b1) of the passes of a length-2^lg transform, lowest first:
// the lowest pass takes up to NTT_TILE_LOG bits (contiguous segments), the
// others up to NTT_TILE_LOG - 5 (tiles of 32 consecutive columns).
inline std::vector<std::pair<int, int>> ntt_passes(int lg) {
    std::vector<std::pair<int, int>> out;
    int b0 = 0;
    while (b0 < lg) {
        const int room = b0 == 0 ? NTT_TILE_LOG : NTT_TILE_LOG - (b0 < 5 ? b0 : 5);
        const int b1 = std::min(lg, b0 + room);
        out.emplace_back(b0, b1);
        b0 = b1;
    }
    return out;
}

// pointwise: C_f = A_f B_f (r x s times s x t) at every transform point f.
// A thread owns one transform point f (consecutive f across a warp, so every
// load is one coalesced row segment) and a PW_RT x PW_CT tile of C; a
// block's eight warps take eight tiles of
// the same 32 points.  The sums sum_k A_ik B_kj run on 64-bit accumulators
// (one 32 x 32 + 64-bit multiply-add per product) folded by 2^32 = r1 (mod P)
// every FOLDK products, reduced mod P and brought to Montgomery form
// (A_ik B_kj R^-1) once at the end.
constexpr int PW_RT = 4, PW_CT = 8, PW_WARPS = 8;

template <int FOLDK>
__global__ void __launch_bounds__(32 * PW_WARPS)
    k_ntt_pointwise_tiled(const uint32_t *__restrict__ A, const uint32_t *__restrict__ B, uint32_t *__restrict__ C,
                          int r, int s, int t, int64_t Lz, ModP mP) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t f = (int64_t)blockIdx.x * 32 + lane;
    const int ntj = (t + PW_CT - 1) / PW_CT, nti = (r + PW_RT - 1) / PW_RT;
    const int tile = blockIdx.y * PW_WARPS + warp;
    if (tile >= nti * ntj || f >= Lz) return;
    const int i0 = (tile / ntj) * PW_RT, j0 = (tile % ntj) * PW_CT;
    const uint32_t fc = mP.r1;  // 2^32 mod P
    bool iv[PW_RT], jv[PW_CT];
    const uint32_t *pa[PW_RT];
    const uint32_t *pb[PW_CT];
#pragma unroll
    for (int u = 0; u < PW_RT; u++) {
        iv[u] = i0 + u < r;
        pa[u] = A + ((size_t)(iv[u] ? i0 + u : 0) * s) * Lz + f;  // row i0 + u, k = 0
    }
#pragma unroll
    for (int v = 0; v < PW_CT; v++) {
        jv[v] = j0 + v < t;
        pb[v] = B + (size_t)(jv[v] ? j0 + v : 0) * Lz + f;  // column j0 + v, k = 0
    }
    const size_t bstep = (size_t)t * Lz;
    unsigned long long acc[PW_RT][PW_CT];
#pragma unroll
    for (int u = 0; u < PW_RT; u++)
#pragma unroll
        for (int v = 0; v < PW_CT; v++) acc[u][v] = 0ull;
    int k = 0;
    for (; k + FOLDK <= s; k += FOLDK) {
#pragma unroll
        for (int kk = 0; kk < FOLDK; kk++) {
            uint32_t a[PW_RT], b[PW_CT];
#pragma unroll
            for (int u = 0; u < PW_RT; u++) a[u] = iv[u] ? __ldg(pa[u] + (size_t)(k + kk) * Lz) : 0u;
#pragma unroll
            for (int v = 0; v < PW_CT; v++) b[v] = jv[v] ? __ldg(pb[v] + (size_t)(k + kk) * bstep) : 0u;
#pragma unroll
            for (int u = 0; u < PW_RT; u++)
#pragma unroll
                for (int v = 0; v < PW_CT; v++) acc[u][v] = madw(a[u], b[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < PW_RT; u++)
#pragma unroll
            for (int v = 0; v < PW_CT; v++) acc[u][v] = fold2(acc[u][v], fc);
    }
    for (; k < s; k++) {  // fewer than FOLDK products after the last fold
        uint32_t a[PW_RT], b[PW_CT];
#pragma unroll
        for (int u = 0; u < PW_RT; u++) a[u] = iv[u] ? __ldg(pa[u] + (size_t)k * Lz) : 0u;
#pragma unroll
        for (int v = 0; v < PW_CT; v++) b[v] = jv[v] ? __ldg(pb[v] + (size_t)k * bstep) : 0u;
#pragma unroll
        for (int u = 0; u < PW_RT; u++)
#pragma unroll
            for (int v = 0; v < PW_CT; v++) acc[u][v] = madw(a[u], b[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < PW_RT; u++)
#pragma unroll
        for (int v = 0; v < PW_CT; v++)
            if (iv[u] && jv[v]) C[((size_t)(i0 + u) * t + j0 + v) * Lz + f] = mont_redc(red64(acc[u][v], mP), mP);
}

struct CrtConst {
    uint32_t P1, P2, P3;
    uint32_t c12;        // P1^{-1} mod P2
    uint32_t c123;       // (P1 P2)^{-1} mod P3
    uint32_t p1_mod_p3;  // P1 mod P3
    uint32_t P1_mod_p, P1P2_mod_p;
};

// Garner: the integer x < P1 P2 P3 with x = r_i mod P_i, reduced mod p.
// In: the three inverse transforms (Montgomery form, still times Lz), one
// run of Lz coefficients per entry; out: coefficient-major.  Tiles of 32
// coefficients x 32 entries: coalesced reads along the coefficients of an
// entry, Garner in registers, a shared-memory transpose, coalesced writes
// along the entries of a coefficient.
__global__ void __launch_bounds__(TR_TILE * TR_ROWS)
    k_ntt_crt(const uint32_t *__restrict__ R1, const uint32_t *__restrict__ R2, const uint32_t *__restrict__ R3,
              int nent, int64_t Lz, int64_t lo, int64_t hi, uint32_t *__restrict__ out, uint32_t il1, uint32_t il2,
              uint32_t il3, CrtConst cc, ModP m1, ModP m2, ModP m3, ModP mp) {
    __shared__ uint32_t tile[TR_TILE][TR_TILE + 1];
    const int tx = threadIdx.x & (TR_TILE - 1), ty = threadIdx.x / TR_TILE;
    const int64_t nk = hi - lo;
    const int64_t ktiles = (nk + TR_TILE - 1) / TR_TILE, etiles = (nent + TR_TILE - 1) / TR_TILE;
    for (int64_t tl = blockIdx.x; tl < ktiles * etiles; tl += gridDim.x) {
        const int64_t k0 = lo + (tl % ktiles) * TR_TILE;
        const int e0 = (int)(tl / ktiles) * TR_TILE;
        __syncthreads();
        for (int y = ty; y < TR_TILE; y += TR_ROWS) {
            const int e = e0 + y;
            const int64_t k = k0 + tx;
            uint32_t v = 0;
            if (e < nent && k < hi) {
                const size_t src = (size_t)e * Lz + (size_t)k;
                // mont_mul(v R, Lz^{-1}) = v Lz^{-1} in normal form
                const uint32_t r1 = mont_mul(R1[src], il1, m1);
                const uint32_t r2 = mont_mul(R2[src], il2, m2);
                const uint32_t r3 = mont_mul(R3[src], il3, m3);
                const uint32_t t1 = r1;
                const uint32_t t2 = mulm(subm(r2, t1 % cc.P2, m2), cc.c12, m2);
                uint32_t u = subm(r3, t1 % cc.P3, m3);
                u = subm(u, mulm(cc.p1_mod_p3, t2, m3), m3);
                const uint32_t t3 = mulm(u, cc.c123, m3);
                uint64_t w = (uint64_t)(t1 % mp.p);
                w += (uint64_t)mulm(cc.P1_mod_p, t2 % mp.p, mp);
                w += (uint64_t)mulm(cc.P1P2_mod_p, t3 % mp.p, mp);
                v = red64(w, mp);
            }
            tile[y][tx] = v;
        }
        __syncthreads();
        for (int y = ty; y < TR_TILE; y += TR_ROWS) {
            const int64_t k = k0 + y;
            const int e = e0 + tx;
            if (k < hi && e < nent) out[(size_t)(k - lo) * nent + e] = tile[tx][y];
        }
    }
}

// blocks of the tiled transposes: one per 32 x 32 tile, at most 16 per SM
// (grid-stride beyond)
inline unsigned tr_grid(int64_t nk, int64_t nent, int num_sms) {
    const int64_t tiles = ((nk + TR_TILE - 1) / TR_TILE) * ((nent + TR_TILE - 1) / TR_TILE);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms * 16));
}

}  // namespace

// The context's twiddle tables, kept across products: for each transform
// prime, the powers w^j and w^-j (j < 2^(LG-1)) of a 2^LG-th root of unity,
// LG >= lg (a shorter transform takes every 2^(LG-lg)-th entry); built on
// the device when a longer transform than the tables serve is first needed.
static wr_status ensure_twiddles(wr_ctx *ctx, int lg) {
    if (ctx->ntt_lg >= lg) return WR_OK;
    const int LG = std::max(lg, 14);
    const int64_t half = (int64_t)1 << (LG - 1);
    WR_TRY(dev_alloc(ctx, ctx->ntt_tw, sizeof(uint32_t) * (size_t)(2 * NTT_NPRIMES) * half));
    for (int i = 0; i < NTT_NPRIMES; i++) {
        const uint32_t P = NTT_PRIMES[i];
        const ModP mP = make_modp(P);
        const uint64_t g = primitive_root(P);
        const uint64_t w = hpow(g, (P - 1) >> LG, P), wi = hpow(w, P - 2, P);
        const uint32_t wm = (uint32_t)(((unsigned __int128)w << 32) % P), wim = (uint32_t)(((unsigned __int128)wi << 32) % P);
        uint32_t *tw = ctx->ntt_tw.as<uint32_t>() + (size_t)(2 * i) * half;
        const unsigned g2 = (unsigned)std::min<int64_t>((half + 255) / 256, (int64_t)ctx->num_sms * 16);
        k_twiddles<<<g2, 256, 0, ctx->stream>>>(wm, half, tw, mP);
        WR_LAUNCHED(ctx);
        k_twiddles<<<g2, 256, 0, ctx->stream>>>(wim, half, tw + half, mP);
        WR_LAUNCHED(ctx);
    }
    ctx->ntt_lg = LG;
    return WR_OK;
}

// C[k - lo] = sum_j A_j B_{k-j} (mod p) for lo <= k < hi; A: na coefficients of
// r x s, B: nb coefficients of s x t, C: (hi - lo) x r x t.  All device
// pointers, coefficient-major.
static wr_status polymat_mul_run(wr_ctx *ctx, const uint32_t *A, int64_t na, const uint32_t *B, int64_t nb, int r,
                                 int s, int t, int64_t lo, int64_t hi, uint32_t p, uint32_t *C);

wr_status polymat_mul(wr_ctx *ctx, const uint32_t *A, int64_t na, const uint32_t *B, int64_t nb, int r, int s,
                      int t, int64_t lo, int64_t hi, uint32_t p, uint32_t *C) {
    if (!ctx->profiling) return polymat_mul_run(ctx, A, na, B, nb, r, s, t, lo, hi, p, C);
    // profiling: the product's device time, summed over the sigma-basis
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    WR_CUDA(cudaEventCreate(&e0));
    WR_CUDA(cudaEventCreate(&e1));
    WR_CUDA(cudaEventRecord(e0, ctx->stream));
    const wr_status st = polymat_mul_run(ctx, A, na, B, nb, r, s, t, lo, hi, p, C);
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ctx->last.sigma_product_ms += ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

static wr_status polymat_mul_run(wr_ctx *ctx, const uint32_t *A, int64_t na, const uint32_t *B, int64_t nb, int r,
                                 int s, int t, int64_t lo, int64_t hi, uint32_t p, uint32_t *C) {
    if (hi <= lo) return WR_OK;
    cudaStream_t st = ctx->stream;
    if (na <= 0 || nb <= 0) {
        WR_CUDA(cudaMemsetAsync(C, 0, sizeof(uint32_t) * (size_t)(hi - lo) * r * t, st));
        return WR_OK;
    }
    // the exact coefficients, at most s min(na, nb) (p - 1)^2, must lie below
    // the product of the transform primes for the remainder step to recover them
    const double bound = (double)s * (double)std::min(na, nb) * (double)(p - 1) * (double)(p - 1);
    if (bound >= 0.999 * (double)NTT_PRIMES[0] * (double)NTT_PRIMES[1] * (double)NTT_PRIMES[2])
        return fail(WR_EINVAL, "polynomial product coefficients exceed the transform primes' product");
    const int64_t full = na + nb - 1;  // coefficients of the exact product
    const int64_t need = std::max<int64_t>(hi, full - lo);
    int lg = 1;
    while (((int64_t)1 << lg) < need) lg++;
    if (lg > NTT_MAX_LOG) return fail(WR_EINVAL, "polynomial product too long for the transform primes");
    const int64_t Lz = (int64_t)1 << lg;
    const int nA = r * s, nB = s * t, nC = r * t;
    const ModP mp = make_modp(p);
    DevBuf bufA, bufB, bufC[NTT_NPRIMES];
    WR_TRY(dev_alloc(ctx, bufA, sizeof(uint32_t) * (size_t)nA * Lz));
    WR_TRY(dev_alloc(ctx, bufB, sizeof(uint32_t) * (size_t)nB * Lz));
    for (int i = 0; i < NTT_NPRIMES; i++) WR_TRY(dev_alloc(ctx, bufC[i], sizeof(uint32_t) * (size_t)nC * Lz));
    WR_TRY(ensure_twiddles(ctx, lg));
    const int LG = ctx->ntt_lg, tshift = LG - lg;  // the length-2^lg twiddle j is table entry j << tshift
    uint32_t il[NTT_NPRIMES];
    ModP mP[NTT_NPRIMES];
    for (int i = 0; i < NTT_NPRIMES; i++) {
        const uint32_t P = NTT_PRIMES[i];
        mP[i] = make_modp(P);
        const uint32_t *tw = ctx->ntt_tw.as<uint32_t>() + (size_t)(2 * i) * ((size_t)1 << (LG - 1));
        const uint32_t *twi = tw + ((size_t)1 << (LG - 1));
        il[i] = (uint32_t)hpow((uint64_t)(Lz % P), P - 2, P);  // Lz^{-1} mod P (normal form)
        k_ntt_load<<<tr_grid(Lz, nA, ctx->num_sms), TR_TILE * TR_ROWS, 0, st>>>(A, na, nA, Lz, bufA.as<uint32_t>(), mP[i]);
        WR_LAUNCHED(ctx);
        k_ntt_load<<<tr_grid(Lz, nB, ctx->num_sms), TR_TILE * TR_ROWS, 0, st>>>(B, nb, nB, Lz, bufB.as<uint32_t>(), mP[i]);
        WR_LAUNCHED(ctx);
        const auto passes = ntt_passes(lg);
        const int tile_log = NTT_TILE_LOG;
        auto pass_grid = [&](int64_t npoly) {
            const int64_t tiles = npoly * (Lz >> std::min<int64_t>(lg, tile_log));
            return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)ctx->num_sms * 8));
        };
        for (auto it = passes.rbegin(); it != passes.rend(); ++it) {  // forward: highest bits first
            k_ntt_pass<true><<<pass_grid(nA), NTT_PASS_THREADS, 0, st>>>(bufA.as<uint32_t>(), nA, lg, it->first,
                                                                        it->second, tw, tshift, mP[i]);
            WR_LAUNCHED(ctx);
            k_ntt_pass<true><<<pass_grid(nB), NTT_PASS_THREADS, 0, st>>>(bufB.as<uint32_t>(), nB, lg, it->first,
                                                                        it->second, tw, tshift, mP[i]);
            WR_LAUNCHED(ctx);
        }
        {
            const int fk = fold_products(NTT_PRIMES[i]);
            auto *kpw = fk >= 14 ? k_ntt_pointwise_tiled<14> : (fk >= 4 ? k_ntt_pointwise_tiled<4> : k_ntt_pointwise_tiled<2>);
            const int tiles = ((r + PW_RT - 1) / PW_RT) * ((t + PW_CT - 1) / PW_CT);
            const dim3 g((unsigned)((Lz + 31) / 32), (unsigned)((tiles + PW_WARPS - 1) / PW_WARPS));
            kpw<<<g, 32 * PW_WARPS, 0, st>>>(bufA.as<uint32_t>(), bufB.as<uint32_t>(), bufC[i].as<uint32_t>(), r, s,
                                              t, Lz, mP[i]);
            WR_LAUNCHED(ctx);
        }
        for (const auto &ps : passes) {  // inverse: lowest bits first
            k_ntt_pass<false><<<pass_grid(nC), NTT_PASS_THREADS, 0, st>>>(bufC[i].as<uint32_t>(), nC, lg, ps.first,
                                                                         ps.second, twi, tshift, mP[i]);
            WR_LAUNCHED(ctx);
        }
    }
    CrtConst cc;
    cc.P1 = NTT_PRIMES[0];
    cc.P2 = NTT_PRIMES[1];
    cc.P3 = NTT_PRIMES[2];
    cc.c12 = (uint32_t)hpow(cc.P1 % cc.P2, cc.P2 - 2, cc.P2);
    cc.c123 = (uint32_t)hpow((uint64_t)cc.P1 * cc.P2 % cc.P3, cc.P3 - 2, cc.P3);
    cc.p1_mod_p3 = cc.P1 % cc.P3;
    cc.P1_mod_p = cc.P1 % p;
    cc.P1P2_mod_p = (uint32_t)((uint64_t)cc.P1 * cc.P2 % p);
    k_ntt_crt<<<tr_grid(hi - lo, nC, ctx->num_sms), TR_TILE * TR_ROWS, 0, st>>>(
        bufC[0].as<uint32_t>(), bufC[1].as<uint32_t>(), bufC[2].as<uint32_t>(), nC, Lz, lo, hi, C, il[0], il[1],
        il[2], cc, mP[0], mP[1], mP[2], mp);
    WR_LAUNCHED(ctx);
    return WR_OK;
}

}  // namespace wr
