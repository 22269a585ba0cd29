// The SpMM pass kernel of the black box (Section 2.5 step 2: the sparse
// products A T and A^T W mod p) and its helpers: SELL-C-sigma light chunks
// and warp-per-segment long rows, exact int64 row sums, the diagonal scaling
// and Montgomery reduction as the epilogue, split rows finished by
// k_finalize_split.  Included by wr_spmm.cu only (its launchers and the
// sequence loop live there).
#pragma once

#include <cuda_runtime.h>

#include "wr_internal.cuh"

namespace wr {
namespace {

// W residues per lane, G lanes per gathered row: one warp-wide gather then
// touches 32/G rows, each one contiguous 4*NV-byte run, so the L1 handles one
// tag lookup per row instead of one per lane.  Random gathers of 32-byte rows
// from an L2-resident table run fastest as 4 lanes of 8 bytes (measured on
// GB300: 10-15% ahead of 2 lanes of 16 bytes, well ahead of one lane of 32
// bytes); rows of 64 bytes and more take 16 bytes per lane.
template <int NV, int WW = (NV <= 8 ? (NV < 2 ? NV : 2) : 4)>
struct Lanes {
    static constexpr int W = WW;       // residues per lane
    static constexpr int G = NV / W;   // lanes per row
    static constexpr int RPW = 32 / G; // rows (light) or entries (vector) per warp step
    static_assert(NV % W == 0 && G >= 1 && G <= 32, "lane width must divide the block width");
};
// default residues per lane for a block width (used when nothing is tuned)
inline int default_lane_width(int nv) { return nv <= 8 ? (nv < 2 ? nv : 2) : 4; }

template <int W>
__device__ __forceinline__ void ldv(const uint32_t *p, uint32_t (&v)[W]) {
    if constexpr (W == 1) {
        v[0] = __ldg(p);
    } else if constexpr (W == 2) {
        uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
        v[0] = t.x; v[1] = t.y;
    } else {
#pragma unroll
        for (int k = 0; k < W / 4; k++) {
            uint4 t = __ldg(reinterpret_cast<const uint4 *>(p) + k);
            v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
        }
    }
}

template <int W>
__device__ __forceinline__ void stv(uint32_t *p, const uint32_t (&v)[W]) {
    if constexpr (W == 1) {
        p[0] = v[0];
    } else if constexpr (W == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1]);
    } else {
#pragma unroll
        for (int k = 0; k < W / 4; k++)
            reinterpret_cast<uint4 *>(p)[k] = make_uint4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
}

// W residues from memory this kernel also writes (the partial output of the
// previous column slab): plain loads
template <int W>
__device__ __forceinline__ void ldv_rw(const uint32_t *p, uint32_t (&v)[W]) {
    if constexpr (W == 1) {
        v[0] = p[0];
    } else if constexpr (W == 2) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
#pragma unroll
        for (int k = 0; k < W / 4; k++) {
            const uint4 t = reinterpret_cast<const uint4 *>(p)[k];
            v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
        }
    }
}

// Loads of the matrix's entry words and stores of the output rows, with or
// without the streaming cache hint (CS: evict-first in L1 and L2, ld/st.cs):
// each entry and each output row is touched once per pass, so with the hint
// they stop pushing rows of the gathered block out of L2.  The autotuner
// times both forms per matrix.
template <bool CS>
__device__ __forceinline__ uint32_t lde(const uint32_t *p) {
    if constexpr (CS) return __ldcs(p);
    else return __ldg(p);
}

template <int W, bool CS>
__device__ __forceinline__ void stv_out(uint32_t *p, const uint32_t (&v)[W]) {
    if constexpr (!CS) {
        stv<W>(p, v);
    } else if constexpr (W == 1) {
        __stcs(p, v[0]);
    } else if constexpr (W == 2) {
        __stcs(reinterpret_cast<uint2 *>(p), make_uint2(v[0], v[1]));
    } else {
#pragma unroll
        for (int k = 0; k < W / 4; k++)
            __stcs(reinterpret_cast<uint4 *>(p) + k, make_uint4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
    }
}

// Entry words: (column << 8) | (uint8)value in the packed layout, the column
// alone in the wide one (values from the int16 array beside the entries).
template <bool WIDE>
__device__ __forceinline__ uint32_t entry_col(uint32_t e) { return WIDE ? e : (e >> 8); }
template <bool WIDE>
__device__ __forceinline__ int entry_val(uint32_t e, const int16_t *wv, int64_t idx) {
    if constexpr (WIDE) return (int)__ldg(wv + idx);
    else return (int)(int8_t)(e & 0xFFu);
}

template <int W>
__device__ __forceinline__ void mac(int64_t (&acc)[W], int a, const uint32_t (&v)[W]) {
#pragma unroll
    for (int w = 0; w < W; w++) acc[w] += (int64_t)a * (int32_t)v[w];
}

// Epilogue of a finished row: y[row] = scale[row] * (sum mod p), or, for a
// row cut into segments, the exact partial sums added into acc64.
// A direct row has at most VSEG = 256 entries of magnitude below 2^15, so
// |sum| < 2^23 p and T = sum + 2^23 p lies in [0, 2^24 p), below p R: one
// Montgomery reduction gives T R^{-1}; with the scale taken to scale R^2 mod p
// (two Montgomery products), mont_mul(T R^{-1}, scale R^2) = sum * scale mod p.
// the modulus and scale of the job owning columns col0.. of a multi-job block
__device__ __forceinline__ void job_of(const MultiEpi &me, int col0, ModP &mp, const uint32_t *&scale) {
    switch (col0 >> me.jw_log) {
        case 0: mp = me.mp[0]; scale = me.scale[0]; break;
        case 1: mp = me.mp[1]; scale = me.scale[1]; break;
        case 2: mp = me.mp[2]; scale = me.scale[2]; break;
        default: mp = me.mp[3]; scale = me.scale[3]; break;
    }
}

// part: 0 the whole pass (y = scale (A x)); with column slabs of the matrix
// (passes split by ranges of the gathered rows, so that the rows of x that a
// slab gathers stay in L2) 1 the first slab (y = its sum mod p), 2 a middle
// one (y += its sum), 3 the last (y = scale (y + its sum)); y holds residues
// in between.
template <int W, bool CS, bool MULTI>
__device__ __forceinline__ void row_out(uint32_t tgt, const int64_t (&acc)[W], uint32_t *y,
                                        const uint32_t *scale_one, unsigned long long *acc64, int nv,
                                        int col0, const ModP &mp_one, const MultiEpi &me, int part) {
    ModP mp = mp_one;
    const uint32_t *scale = scale_one;
    if constexpr (MULTI) {
        if (!(tgt & VROW_SPLIT)) job_of(me, col0, mp, scale);
    }
    if (tgt & VROW_SPLIT) {
        unsigned long long *dst = acc64 + (size_t)(tgt & ~VROW_SPLIT) * nv + col0;
#pragma unroll
        for (int w = 0; w < W; w++) atomicAdd(dst + w, (unsigned long long)acc[w]);
    } else {
        const uint64_t off = (uint64_t)mp.p << 23;
        uint32_t o[W];
        uint32_t *yr = y + (size_t)tgt * nv + col0;
        if (part == 0) {
            const uint32_t s2 = to_mont(to_mont(__ldg(scale + tgt), mp), mp);
#pragma unroll
            for (int w = 0; w < W; w++) o[w] = mont_mul(mont_redc((uint64_t)acc[w] + off, mp), s2, mp);
        } else {
            // mont_mul(T R^{-1}, R^2) = T mod p
#pragma unroll
            for (int w = 0; w < W; w++) o[w] = mont_mul(mont_redc((uint64_t)acc[w] + off, mp), mp.r2, mp);
            if (part >= 2) {
                uint32_t prev[W];
                ldv_rw<W>(yr, prev);
#pragma unroll
                for (int w = 0; w < W; w++) o[w] = addm(o[w], prev[w], mp);
            }
            if (part == 3) {
                const uint32_t s1 = to_mont(__ldg(scale + tgt), mp);
#pragma unroll
                for (int w = 0; w < W; w++) o[w] = mont_mul(o[w], s1, mp);
            }
        }
        stv_out<W, CS>(yr, o);
    }
}

// One SpMM pass, y = scale * (A x) mod p, exact int64 row sums.
// Blocks [0, vblocks): one warp per segment of a long row; its lanes stride
// over the segment's contiguous entries, then a shuffle reduction.
// Blocks [vblocks, ...): G warps per SELL chunk of 32 light rows; warp q of
// the chunk takes rows [q*RPW, (q+1)*RPW), G lanes per row.
template <int NV, int WL, bool WIDE, bool CS, bool MULTI>
__global__ void __launch_bounds__(256) k_spmm(SellView A, const uint32_t *__restrict__ x,
                                              uint32_t *__restrict__ y,
                                              const uint32_t *__restrict__ scale,
                                              unsigned long long *__restrict__ acc64, ModP mp,
                                              int *__restrict__ term_counter, int64_t vblocks, MultiEpi me,
                                              int part) {
    using Ln = Lanes<NV, WL>;
    constexpr int W = Ln::W, G = Ln::G, RPW = Ln::RPW;
    if (term_counter && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(term_counter, 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / G, lanepart = lane % G;
    const uint32_t *xb = x + lanepart * W;
    if ((int64_t)blockIdx.x < vblocks) {
        const int64_t seg = (int64_t)blockIdx.x * 8 + warp;
        if (seg >= A.nseg) return;
        const uint32_t *e = A.ventries + A.seg_start[seg];
        const int16_t *ev = WIDE ? A.vwvals + A.seg_start[seg] : nullptr;
        const int len = A.seg_len[seg];
        int64_t acc[W];
#pragma unroll
        for (int w = 0; w < W; w++) acc[w] = 0;
        int j = sub;
        for (; j + 3 * RPW < len; j += 4 * RPW) {
            const uint32_t e0 = lde<CS>(e + j), e1 = lde<CS>(e + j + RPW);
            const uint32_t e2 = lde<CS>(e + j + 2 * RPW), e3 = lde<CS>(e + j + 3 * RPW);
            uint32_t v0[W], v1[W], v2[W], v3[W];
            ldv<W>(xb + (size_t)entry_col<WIDE>(e0) * NV, v0);
            ldv<W>(xb + (size_t)entry_col<WIDE>(e1) * NV, v1);
            ldv<W>(xb + (size_t)entry_col<WIDE>(e2) * NV, v2);
            ldv<W>(xb + (size_t)entry_col<WIDE>(e3) * NV, v3);
            mac<W>(acc, entry_val<WIDE>(e0, ev, j), v0);
            mac<W>(acc, entry_val<WIDE>(e1, ev, j + RPW), v1);
            mac<W>(acc, entry_val<WIDE>(e2, ev, j + 2 * RPW), v2);
            mac<W>(acc, entry_val<WIDE>(e3, ev, j + 3 * RPW), v3);
        }
        for (; j < len; j += RPW) {
            const uint32_t e0 = lde<CS>(e + j);
            uint32_t v0[W];
            ldv<W>(xb + (size_t)entry_col<WIDE>(e0) * NV, v0);
            mac<W>(acc, entry_val<WIDE>(e0, ev, j), v0);
        }
#pragma unroll
        for (int off = G; off < 32; off <<= 1)
#pragma unroll
            for (int w = 0; w < W; w++) acc[w] += __shfl_xor_sync(0xffffffffu, acc[w], off);
        if (sub == 0) row_out<W, CS, MULTI>(A.seg_row[seg], acc, y, scale, acc64, NV, lanepart * W, mp, me, part);
        return;
    }
    const int64_t lw = ((int64_t)blockIdx.x - vblocks) * 8 + warp;
    const int64_t chunk = lw / G;
    if (chunk >= A.nchunks) return;
    const int64_t base = A.chunk_off[chunk];
    const int len = A.chunk_len[chunk];
    {
        const int r = (int)(lw % G) * RPW + sub;
        const uint32_t *e = A.entries + base + r;
        const int16_t *ev = WIDE ? A.wvals + base + r : nullptr;
        int64_t acc[W];
#pragma unroll
        for (int w = 0; w < W; w++) acc[w] = 0;
        int j = 0;
        for (; j + 8 <= len; j += 8) {
            uint32_t ee[8];
#pragma unroll
            for (int u = 0; u < 8; u++) ee[u] = lde<CS>(e + (j + u) * SELL_C);
            uint32_t vv[8][W];
#pragma unroll
            for (int u = 0; u < 8; u++) ldv<W>(xb + (size_t)entry_col<WIDE>(ee[u]) * NV, vv[u]);
#pragma unroll
            for (int u = 0; u < 8; u++) mac<W>(acc, entry_val<WIDE>(ee[u], ev, (int64_t)(j + u) * SELL_C), vv[u]);
        }
        for (; j + 4 <= len; j += 4) {
            const uint32_t e0 = lde<CS>(e + (j + 0) * SELL_C), e1 = lde<CS>(e + (j + 1) * SELL_C);
            const uint32_t e2 = lde<CS>(e + (j + 2) * SELL_C), e3 = lde<CS>(e + (j + 3) * SELL_C);
            uint32_t v0[W], v1[W], v2[W], v3[W];
            ldv<W>(xb + (size_t)entry_col<WIDE>(e0) * NV, v0);
            ldv<W>(xb + (size_t)entry_col<WIDE>(e1) * NV, v1);
            ldv<W>(xb + (size_t)entry_col<WIDE>(e2) * NV, v2);
            ldv<W>(xb + (size_t)entry_col<WIDE>(e3) * NV, v3);
            mac<W>(acc, entry_val<WIDE>(e0, ev, (int64_t)(j + 0) * SELL_C), v0);
            mac<W>(acc, entry_val<WIDE>(e1, ev, (int64_t)(j + 1) * SELL_C), v1);
            mac<W>(acc, entry_val<WIDE>(e2, ev, (int64_t)(j + 2) * SELL_C), v2);
            mac<W>(acc, entry_val<WIDE>(e3, ev, (int64_t)(j + 3) * SELL_C), v3);
        }
        for (; j < len; j++) {
            const uint32_t e0 = lde<CS>(e + j * SELL_C);
            uint32_t v0[W];
            ldv<W>(xb + (size_t)entry_col<WIDE>(e0) * NV, v0);
            mac<W>(acc, entry_val<WIDE>(e0, ev, (int64_t)j * SELL_C), v0);
        }
        const uint32_t vr = A.vrow[chunk * SELL_C + r];
        if (vr != VROW_EMPTY) row_out<W, CS, MULTI>(vr, acc, y, scale, acc64, NV, lanepart * W, mp, me, part);
    }
}

// Rows that were cut into segments: their exact int64 sums were added into
// acc64; reduce, scale, store, and clear the accumulator for the next pass.
// (part: as in row_out)
__global__ void k_finalize_split(int64_t nsplit, int nv, const int32_t *__restrict__ split_row,
                                 unsigned long long *__restrict__ acc64, uint32_t *__restrict__ y,
                                 const uint32_t *__restrict__ scale, ModP mp, int part) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsplit * nv) return;
    int64_t sid = i / nv;
    int b = (int)(i % nv);
    int32_t r = split_row[sid];
    unsigned long long s = acc64[i];
    acc64[i] = 0;
    uint32_t *yr = y + (size_t)r * nv + b;
    uint32_t v = red_s64((int64_t)s, mp);
    if (part >= 2) v = addm(v, *yr, mp);
    if (part == 0 || part == 3) v = mulm(scale[r], v, mp);
    *yr = v;
}

// the same for a multi-job block: column b is reduced with its job's modulus and scale
__global__ void k_finalize_split_multi(int64_t nsplit, int nv, const int32_t *__restrict__ split_row,
                                       unsigned long long *__restrict__ acc64, uint32_t *__restrict__ y, MultiEpi me) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsplit * nv) return;
    int64_t sid = i / nv;
    int b = (int)(i % nv);
    int32_t r = split_row[sid];
    unsigned long long s = acc64[i];
    acc64[i] = 0;
    ModP mp;
    const uint32_t *scale;
    job_of(me, b, mp, scale);
    y[(size_t)r * nv + b] = mulm(scale[r], red_s64((int64_t)s, mp), mp);
}

}  // namespace
}  // namespace wr
