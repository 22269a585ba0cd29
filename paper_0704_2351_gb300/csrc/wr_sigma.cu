// sigma-basis of the block Wiedemann sequence and the rank readout
// (Section 2.4 "sigma-basis computations", Section 2.5 steps 3 and 4).
//
// M-Basis (Giorgi, Jeannerod, Villard) computes an order-L sigma-basis M(x)
// of H(x) = [S(x) | -I_m] (m x q, q = m + n) for the shift (0^n, 1^m), one
// order at a time: the discrepancy Delta_k (coefficient k of H M) is
// column-reduced in order of (shifted degree, index), each column by the
// pivots found before it (pivot row = first nonzero row), and the pivot
// columns are multiplied by x.
//
// On the device the orders are processed in chunks of b:
//   window : E_i = coeff_{k0+i}(S P) - [i = 0] Qtop for i < b  (many blocks),
//            where P = first n rows of M and Qtop = coefficient k0 of the
//            last m rows (the only coefficient of those rows that can still
//            matter: their degree is below the shifted degree <= k0 + 1);
//   local  : the b orders of M-Basis on the window alone, building the
//            chunk's transform Mloc (q x q, degree <= b)  (one block);
//   apply  : P <- P Mloc  (many blocks).
// The transforms are those of the order-by-order algorithm (the product of
// the same elementary steps), so P and the degrees are bit-identical to it.
// The elimination runs fraction-free (col_j <- d_c col_j - d_j col_c) and
// divides by the accumulated column scale once per order, which removes the
// modular inverses from the sequential part.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "wr_internal.cuh"

namespace wr {

namespace {

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// The starting basis at x^0.  [S | -I_m] (deg_in == nullptr): P = [I_n | 0]
// (the first n rows), degrees (0^n, 1^m), Q = [0 | I_m].  A general residual
// (deg_in given, nr = q rows): P = I_q, the given degrees, Q = 0.
__global__ void k_init_basis(uint32_t *__restrict__ P, int nr, int n, int q, int32_t *__restrict__ deg,
                             const int32_t *__restrict__ deg_in, uint32_t *__restrict__ qtop, int m,
                             int *__restrict__ dmax) {
    for (int t = threadIdx.x; t < m * q || t < q; t += blockDim.x) {
        if (t < nr) P[(size_t)t * q + t] = 1;
        if (t < q) deg[t] = deg_in ? deg_in[t] : (t < n ? 0 : 1);
        if (t < m * q) {
            int a = t / q, c = t % q;
            qtop[t] = (!deg_in && c == n + a) ? 1u : 0u;
        }
    }
    if (threadIdx.x == 0) *dmax = 1;
}

// Early termination test of one chunk.  The generator candidates are the n
// columns of smallest shifted degree (ties by index); the chunk is quiet when
// each has degree <= k0 (so its -Q part lies below the chunk's orders and the
// window's E is its whole discrepancy) and zero discrepancy at every order of
// the chunk.  Such columns are never touched by the chunk's eliminations.
// *count: consecutive quiet orders so far, mirrored to a host-mapped slot.
__global__ void k_quiet(const uint32_t *__restrict__ E, int bb, int m, int n, int q,
                        const int32_t *__restrict__ deg, int64_t k0, long long *__restrict__ count,
                        long long *host_slot) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < q; c += blockDim.x) {
        const int dc = deg[c];
        int before = 0;
        for (int c2 = 0; c2 < q; c2++) {
            const int d2 = deg[c2];
            before += (d2 < dc || (d2 == dc && c2 < c)) ? 1 : 0;
        }
        if (before >= n) continue;
        bool nz = dc > k0;
        for (int x = 0; x < bb * m && !nz; x++) nz = E[(size_t)x * q + c] != 0u;
        if (nz) atomicOr(&bad, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long v = bad ? 0 : *count + bb;
        *count = v;
        *(volatile long long *)host_slot = v;
    }
}

// ---- window.  Block b takes coefficients t in [b tper, (b+1) tper) and
// writes its partial E_i = sum_t S[k0+i-t] P[t] (mod p) for all i < bb into
// Epart[b]; k_sum_parts adds the partials.
constexpr int WIN_THREADS = 256;
constexpr int WIN_IB = 8;  // orders per thread (IB = 4 for chunks of at most 4 orders)
constexpr int WIN_CB = 4;  // columns per thread
static_assert(WIN_CB == 4, "the 16-byte loads assume tiles of 4 columns");

// Four consecutive residues from shared memory (one 16-byte load when VEC),
// zero where the column is out of range.
template <bool VEC>
__device__ __forceinline__ void ld4(const uint32_t *p, const bool (&cv)[4], uint32_t (&v)[4]) {
    if constexpr (VEC) {
        const uint4 t = *reinterpret_cast<const uint4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = cv[u] ? p[u] : 0u;
    }
}

// Discrepancies of one chunk: E_i = sum_t S_{k0+i-t} P_t for orders
// i < bb (m x q each), the coefficients t of P split over the blocks (each
// writes its partial sums, reduced mod p, to Epart[block]).  A thread owns a
// WIN_IB x WIN_CB tile (orders i0.. x columns c0..) of one row a.  For a fixed
// r it walks the coefficients t of the tile: the S residues the tile needs at
// step t+1 are those of step t shifted by one order, so they live in a
// circular register window that takes one new shared-memory load per step
// (slot indices are compile-time in an IB-fold unrolled loop), and the
// WIN_CB residues of P are one 16-byte load (VEC: q a multiple of 4).
template <int FOLDK, bool VEC, int IB>
__global__ void __launch_bounds__(WIN_THREADS, 1)
    k_window(const uint32_t *__restrict__ S, int64_t L, int m, int n, int q, const uint32_t *__restrict__ P,
             int64_t k0, int bb, int TT, int64_t tper, const int *__restrict__ dmax_dev,
             uint32_t *__restrict__ Epart, ModP mp) {
    extern __shared__ uint32_t sm[];
    const int mn = m * n, nq = n * q, mq = m * q;
    static_assert(IB == 4 || IB == 8, "order tiles of 4 or 8");
    const int nib = (bb + IB - 1) / IB, ncb = (q + WIN_CB - 1) / WIN_CB;
    const int items = nib * m * ncb;
    const uint32_t fc = mp.r1;  // 2^32 mod p
    uint32_t *out = Epart + (size_t)blockIdx.x * bb * mq;
    const int64_t tmax = min64((int64_t)*dmax_dev, k0 + bb - 1);
    const int64_t tb0 = (int64_t)blockIdx.x * tper;
    const int64_t tb1 = min64(tb0 + tper, tmax + 1);
    uint32_t *Ps = sm;                          // [TT][n][q]
    uint32_t *Ss = sm + (size_t)TT * nq;        // [nib*IB + TT - 1][m][n]
    for (int round = 0; round * WIN_THREADS < items; round++) {
        const int it = round * WIN_THREADS + threadIdx.x;
        const bool act = it < items;
        const int cb = act ? it % ncb : 0;
        const int a = act ? (it / ncb) % m : 0;
        const int i0 = act ? (it / (ncb * m)) * IB : 0;
        const int c0 = cb * WIN_CB;
        bool cv[WIN_CB];
#pragma unroll
        for (int u = 0; u < WIN_CB; u++) cv[u] = c0 + u < q;
        Acc2 acc[IB][WIN_CB];
#pragma unroll
        for (int k = 0; k < IB; k++)
#pragma unroll
            for (int u = 0; u < WIN_CB; u++) acc[k][u] = Acc2{0u, 0u};
        int cnt = 0;
        for (int64_t t0 = tb0; t0 < tb1; t0 += TT) {
            const int tt_n = (int)min64(TT, tb1 - t0);
            const int64_t smin = k0 - (t0 + tt_n - 1);
            const int srows = nib * IB + tt_n - 1;
            __syncthreads();
            for (int x = threadIdx.x; x < tt_n * nq; x += WIN_THREADS) Ps[x] = P[(size_t)t0 * nq + x];
            for (int x = threadIdx.x; x < srows * mn; x += WIN_THREADS) {
                const int64_t sidx = smin + x / mn;
                Ss[x] = (sidx >= 0 && sidx < L) ? S[(size_t)sidx * mn + x % mn] : 0u;
            }
            __syncthreads();
            if (!act) continue;
            // order i0+k at coefficient t0+s reads S row smin + (i0 + k + tt_n - 1 - s) = row top - s + k
            const int top = i0 + tt_n - 1;
            for (int r = 0; r < n; r++) {
                const uint32_t *scol = Ss + a * n + r;      // row u at scol[u * mn]
                const uint32_t *pcol = Ps + r * q + c0;     // coefficient s at pcol[s * nq]
                uint32_t sw[IB];                            // row top - s + k in slot (k - s) mod IB
#pragma unroll
                for (int k = 0; k < IB; k++) sw[k] = scol[(size_t)(top + k) * mn];
                for (int s0 = 0; s0 < tt_n; s0 += IB) {
#pragma unroll
                    for (int j = 0; j < IB; j++) {
                        const int st = s0 + j;
                        if (st < tt_n) {
                            if (st > 0) sw[(IB - j) & (IB - 1)] = scol[(size_t)(top - st) * mn];
                            uint32_t pv[WIN_CB];
                            ld4<VEC>(pcol + (size_t)st * nq, cv, pv);
#pragma unroll
                            for (int k = 0; k < IB; k++)
#pragma unroll
                                for (int u = 0; u < WIN_CB; u++) mac2(acc[k][u], sw[(k - j) & (IB - 1)], pv[u]);
                            if (++cnt == FOLDK) {
#pragma unroll
                                for (int k = 0; k < IB; k++)
#pragma unroll
                                    for (int u = 0; u < WIN_CB; u++) fold2w(acc[k][u], fc);
                                cnt = 0;
                            }
                        }
                    }
                }
            }
        }
        if (act) {
#pragma unroll
            for (int k = 0; k < IB; k++) {
                const int i = i0 + k;
#pragma unroll
                for (int u = 0; u < WIN_CB; u++)
                    if (i < bb && cv[u]) out[(size_t)(i * m + a) * q + c0 + u] = red64(acc2_u64(acc[k][u]), mp);
            }
        }
    }
}

// Esum[x] = sum over the window blocks of Epart[b][x], mod p: 32 entries per
// block, 8 groups of blocks per entry, then a shared-memory sum.
__global__ void __launch_bounds__(256)
    k_sum_parts(int nparts, int64_t E, const uint32_t *__restrict__ Epart, uint32_t *__restrict__ Esum, ModP mp) {
    __shared__ unsigned long long red[8][32];
    const int lx = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t x = (int64_t)blockIdx.x * 32 + lx;
    unsigned long long v = 0;  // < 2^31 * nparts
    if (x < E)
        for (int b = g; b < nparts; b += 8) v += __ldg(Epart + (size_t)b * E + x);
    red[g][lx] = v;
    __syncthreads();
    if (g == 0 && x < E) {
#pragma unroll
        for (int k = 1; k < 8; k++) v += red[k][lx];
        Esum[x] = red64(v, mp);
    }
}

// ---- local M-Basis over the window: one block, bb orders.
//
// The device keeps the basis in fraction-free form, M_g = M diag(S): the
// elimination of a discrepancy whose columns are scaled by nonzero constants
// picks the same pivots and yields the same reduced columns up to column
// scales, so M_g stays a column-scaled copy of the order-by-order basis.  S
// (per column, product of the scales of all orders) is divided out of P once
// at the end.
//
// Warp 0 runs the critical path: per order it eliminates the discrepancy with
// one column per lane (q <= 32; k_local_wide takes wider blocks), right-looking and fraction-free in
// Montgomery form -- when the current column (in (degree, index) order) is
// nonzero it becomes a pivot and every later column is reduced by it at once,
// so each column is reduced by exactly the pivots created before it.  It
// publishes the order's transform, new[j] = s_j old[j] + sum_t F[t][j]
// old[pc[t]], and keeps the degree bookkeeping.  The other warps apply the
// transform: first to window rows i and i+1 (the next discrepancy; warp 0
// waits for these), then to rows i+2.., to Qtop (coefficient x^k of the last
// m rows of M) and to the chunk transform Ml.  Named barriers hand the orders
// over: T_i (transform i published; warp 0 arrives, the others wait) and RR_i
// (rows i, i+1 done; the others arrive, warp 0 waits).  Phases alternate
// between two ids per barrier, so a barrier is reused only after its previous
// phase completed: the arrivals of phase k + 2 are ordered after a wait that
// needs phase k complete.  There is no spin-wait.  Multiplying column c by x
// moves no data: window column c is read at row i' - sh[c], and Ml column c
// holds its coefficient s at row base[c] + s; the other warps use per-order
// snapshots of sh and base.
constexpr int LOCAL_THREADS = 1024;
// threads of k_local: all 32 warps for m <= 8; 16 for m > 8; 8 with two
// columns per lane (CPL = 2), so that the elimination warp keeps its columns
// (about 200 residues) in registers
__host__ __device__ constexpr int local_threads(int MM, int CPL) {
    return CPL > 1 ? LOCAL_THREADS / 4 : (MM > 8 ? LOCAL_THREADS / 2 : LOCAL_THREADS);
}
// orders per chunk unless the context sets it (wr_set_sigma_chunk); for
// q > 32 (k_local_wide, whose row work per order grows with the chunk) 4:
// measured at q = 64, L = 8,192, 512-order leaves: 1,678 / 1,518 / 1,299 /
// 1,496 / 1,415 ms for chunks of 2 / 3 / 4 / 5 / 7 orders
constexpr int SIGMA_CHUNK_DEFAULT = 64;
constexpr int SIGMA_CHUNK_WIDE = 4;
// PM-Basis by default only for sequences longer than SIGMA_PM_MIN_L (q <=
// 32), with leaves of SIGMA_LEAF_DEFAULT orders; measured on GB300 at
// L = 45,002, q = 16 the blocked M-Basis alone is faster (744 ms against
// 786-1058 ms for leaves of 16,384 down to 1,024 orders).  For q > 32 the
// M-Basis chunks are a few orders long (shared memory) and the window and
// apply passes over the basis grow with its degree, so PM-Basis with short
// leaves takes over early: at q = 64, L = 8,192, 1,648 / 1,453 / 1,413 ms for
// leaves of 2,048 / 512 / 256 orders, and at L = 118,752 21.5 s with 512
// (46 s with 2,048).  wr_set_sigma_leaf chooses the leaf explicitly.
constexpr int64_t SIGMA_LEAF_DEFAULT = 8192;
constexpr int64_t SIGMA_PM_MIN_L = 131072;
constexpr int64_t SIGMA_LEAF_WIDE = 512;
constexpr int64_t SIGMA_PM_MIN_L_WIDE = 2048;
constexpr int BAR_T0 = 1, BAR_RR0 = 3;  // ids BAR_T0 + (i & 1), BAR_RR0 + (i & 1)

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int nthreads) {
    __threadfence_block();
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The transform of one order held in registers by each lane: for its
// column(s) j, the diagonal dg[j], the coefficients F[t][j] and where the
// pivot columns of the same row live.  apply() computes new[j] = dg[j] old[j]
// + sum_t F[t][j] old[pc[t]] for one row whose column j sits at p[0] (and
// column j + 32 at p[1] when CPL = 2, that is q > 32, one row per warp).
template <int MM, int CPL, int KLAZY>
struct RowTransform {
    uint32_t f[CPL][MM], d[CPL];
    int src[MM];  // CPL = 1: lane holding pc[t]; CPL = 2: pc[t] itself
    int np;

    __device__ __forceinline__ void load(const uint32_t *F, const uint32_t *dg, const int *pcs, int np_, int q,
                                         int W2, int grp, int col, int lane) {
        np = np_;
#pragma unroll
        for (int k = 0; k < CPL; k++) {
            const int j = CPL == 1 ? col : lane + 32 * k;
            d[k] = j < q ? dg[j] : 0u;
#pragma unroll
            for (int t = 0; t < MM; t++) f[k][t] = (t < np && j < q) ? F[t * q + j] : 0u;
        }
#pragma unroll
        for (int t = 0; t < MM; t++) {
            const int c = t < np ? pcs[t] : 0;
            src[t] = CPL == 1 ? grp * W2 + c : c;
        }
    }

    __device__ __forceinline__ void apply(uint32_t *const (&ptr)[CPL], const ModP &mp) const {
        uint32_t v[CPL];
        unsigned long long a[CPL];
#pragma unroll
        for (int k = 0; k < CPL; k++) {
            v[k] = ptr[k] ? *ptr[k] : 0u;
            a[k] = (unsigned long long)d[k] * v[k];
        }
#pragma unroll
        for (int t = 0; t < MM; t++) {
            if (t < np) {
                uint32_t oc;
                if (CPL == 1) {
                    oc = __shfl_sync(0xffffffffu, v[0], src[t]);
                } else {
                    const uint32_t x0 = __shfl_sync(0xffffffffu, v[0], src[t] & 31);
                    const uint32_t x1 = __shfl_sync(0xffffffffu, v[CPL - 1], src[t] & 31);
                    oc = src[t] >= 32 ? x1 : x0;
                }
#pragma unroll
                for (int k = 0; k < CPL; k++) a[k] += (unsigned long long)f[k][t] * oc;
                // at most KLAZY products (plus a reduced residue) between reductions
                if (MM + 1 > KLAZY && (t + 2) % KLAZY == 0) {
#pragma unroll
                    for (int k = 0; k < CPL; k++) a[k] = red64(a[k], mp);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < CPL; k++)
            if (ptr[k]) *ptr[k] = red64(a[k], mp);
    }
};

// Warp 0 of k_local when q <= 16: two lanes per column.  Lane L holds
// column j = L & 15 and half h = L >> 4 of it: discrepancy rows
// h*MM/2 .. h*MM/2 + MM/2 - 1 and the same range of its transform row, so a
// pivot step costs each lane half the Montgomery updates of the one-lane
// layout.  The elimination, the published transform and the bookkeeping are
// those of the one-lane path (same pivots, same fraction-free values).
template <int MM>
__device__ __forceinline__ void local_warp0_two_lane(int m, int q, int bb, const uint32_t *Es, uint32_t *Tb, int tw,
                                                     int *snap, int snapw, int *deg, int *degl, int *sh, int *base,
                                                     uint32_t *scale_g, int nth, const ModP &mp) {
    constexpr int HM = MM / 2;
    const int lane = threadIdx.x & 31;
    const int j = lane & 15, h = lane >> 4;
    const bool v = j < q;
    const int mq = m * q;
    uint32_t scum = mp.r1;  // cumulative column scale over the chunk (Montgomery form)
    for (int i = 0; i < bb; i++) {
        uint32_t *F = Tb + (i & 1) * tw;
        uint32_t *dg = F + mq;
        int *sn = snap + (i & 1) * snapw;
        int *s_sh = sn, *s_base = sn + q, *s_isp = sn + 2 * q, *s_pc = sn + 3 * q;
        uint32_t d[HM], tp[HM], sc = mp.r1;
        int rk = 1 << 20;
        if (v) {
            int r0 = 0;
            const int dj = deg[j];
            for (int c2 = 0; c2 < q; c2++) {
                const int dc2 = deg[c2];
                r0 += (dc2 < dj || (dc2 == dj && c2 < j)) ? 1 : 0;
            }
            rk = r0;
            if (h == 0) {
                s_isp[j] = 0;
                s_sh[j] = sh[j];
                s_base[j] = base[j];
            }
        }
        {
            const uint32_t *er = Es + (size_t)(i - (v ? sh[j] : 0)) * mq + (v ? j : 0);
#pragma unroll
            for (int r = 0; r < HM; r++) {
                const int a2 = h * HM + r;
                d[r] = (v && a2 < m) ? to_mont(er[a2 * q], mp) : 0u;
                tp[r] = 0u;
            }
        }
        int np = 0;
        for (int step = 0; step < q; step++) {
            const bool mine = rk == step;
            const unsigned who = __ballot_sync(0xffffffffu, mine);
            const int src0 = __ffs(who) - 1;  // the h = 0 lane of the current column
            int frl = -1;
            if (mine) {
#pragma unroll
                for (int r = HM - 1; r >= 0; r--)
                    if (d[r] != 0) frl = h * HM + r;
            }
            const int fr0 = __shfl_sync(0xffffffffu, frl, src0);
            const int fr1 = __shfl_sync(0xffffffffu, frl, src0 + 16);
            const int fr = fr0 >= 0 ? fr0 : fr1;
            if (fr < 0) continue;
            const int hp = fr / HM, rp = fr - hp * HM;
            const uint32_t sc_cur = __shfl_sync(0xffffffffu, sc, src0);
            uint32_t pv[HM], pt[HM];
#pragma unroll
            for (int r = 0; r < HM; r++) {
                pv[r] = __shfl_sync(0xffffffffu, d[r], src0 + 16 * h);
                pt[r] = __shfl_sync(0xffffffffu, tp[r], src0 + 16 * h);
            }
            uint32_t x = 0;  // this lane's residue at pivot row offset rp
#pragma unroll
            for (int r = 0; r < HM; r++)
                if (r == rp) x = d[r];
            const uint32_t dc = __shfl_sync(0xffffffffu, x, src0 + 16 * hp);
            const uint32_t dj = __shfl_sync(0xffffffffu, x, j + 16 * hp);
            if (rk > step && rk < (1 << 20) && dj != 0) {
                // col <- dc col - dj pivot: one Montgomery reduction of
                // dc*x + (p - dj)*y < 2 p^2 < p 2^32 per entry
                const uint64_t ndj = mp.p - dj;
#pragma unroll
                for (int r = 0; r < HM; r++) d[r] = mont_redc((uint64_t)dc * d[r] + ndj * pv[r], mp);
#pragma unroll
                for (int r = 0; r < HM; r++) {
                    const int t = h * HM + r;
                    if (t < np) tp[r] = mont_redc((uint64_t)dc * tp[r] + ndj * pt[r], mp);
                    else if (t == np) tp[r] = mont_redc(ndj * sc_cur, mp);
                }
                sc = mont_mul(sc, dc, mp);
            }
            if (lane == 0) {
                s_pc[np] = src0;
                s_isp[src0] = 1;
            }
            np++;
        }
        __syncwarp();
        // publish the transform (normal form) and the local degree bounds
        int dl = 0;
        if (v) {
            dl = degl[j];
#pragma unroll
            for (int r = 0; r < HM; r++) {
                const int t = h * HM + r;
                if (t < np) {
                    const uint32_t val = from_mont(tp[r], mp);
                    F[t * q + j] = val;
                    if (val) dl = max(dl, degl[s_pc[t]]);
                }
            }
            if (h == 0) dg[j] = from_mont(sc, mp);
            scum = mont_mul(scum, sc, mp);
        }
        dl = max(dl, __shfl_xor_sync(0xffffffffu, dl, 16));  // both halves of the column
        int dmx = dl;
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) dmx = max(dmx, __shfl_xor_sync(0xffffffffu, dmx, off));
        if (lane == 0) {
            sn[3 * q + m] = np;
            sn[3 * q + m + 1] = dmx;
        }
        __syncwarp();
        named_arrive(BAR_T0 + (i & 1), nth);
        // ---- bookkeeping of order i: local degrees, pivots times x
        if (v && h == 0) degl[j] = dl;
        __syncwarp();
        for (int t = lane; t < np; t += 32) {
            const int c = s_pc[t];
            deg[c] += 1;
            degl[c] += 1;
            sh[c] += 1;
            base[c] -= 1;
        }
        __syncwarp();
        // ---- the next discrepancy (rows i, i+1) must be done
        named_sync(BAR_RR0 + (i & 1), nth);
    }
    if (v && h == 0) scale_g[j] = mont_mul(scale_g[j], scum, mp);
}

template <int MM, int CPL, int KLAZY>
__global__ void __launch_bounds__(local_threads(MM, CPL))
    k_local(int m, int n, int q, int bb, int nparts, const uint32_t *__restrict__ Epart,
            uint32_t *__restrict__ qtop_g, int32_t *__restrict__ deg_g, uint32_t *__restrict__ Ml_g,
            int32_t *__restrict__ degl_g, int *__restrict__ dmax_g, uint32_t *__restrict__ scale_g, int dbase,
            ModP mp) {
    extern __shared__ uint32_t sm[];
    const int mq = m * q, qq = q * q;
    const int mlrows = 2 * bb + 1;
    const int tw = mq + q;                               // transform: F (m x q) then diagonal (q)
    uint32_t *Es = sm;                                   // bb*m*q
    uint32_t *Ml = Es + (size_t)bb * mq;                 // (2bb+1)*q*q
    uint32_t *Tb = Ml + (size_t)mlrows * qq;             // 2 * tw (double buffer)
    uint32_t *qt = Tb + 2 * tw;                          // m*q
    int *deg = (int *)(qt + mq);                         // q
    int *degl = deg + q;                                 // q
    int *sh = degl + q;                                  // q
    int *base = sh + q;                                  // q
    int *snap = base + q;                                // 2 * snapw: sh, base, isp, pc, np, dl
    const int snapw = 3 * q + m + 2;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    const int E = bb * mq;
    (void)n;

    for (int x = tid; x < mq; x += nth) qt[x] = qtop_g[x];
    __syncthreads();
    for (int x = tid; x < E; x += nth) {
        unsigned long long v = 0;
        int b = 0;
        for (; b + 4 <= nparts; b += 4)
            v += (unsigned long long)Epart[(size_t)b * E + x] + Epart[(size_t)(b + 1) * E + x] +
                 Epart[(size_t)(b + 2) * E + x] + Epart[(size_t)(b + 3) * E + x];
        for (; b < nparts; b++) v += Epart[(size_t)b * E + x];
        uint32_t e = red64(v, mp);
        if (x < mq) e = subm(e, qt[x], mp);
        Es[x] = e;
    }
    for (int x = tid; x < mlrows * qq; x += nth) {
        const int s2 = x / qq, rem = x - s2 * qq;
        Ml[x] = (s2 == bb && rem / q == rem % q) ? 1u : 0u;  // logical coefficient 0 at row base = bb
    }
    for (int c = tid; c < q; c += nth) {
        deg[c] = deg_g[c];
        degl[c] = 0;
        sh[c] = 0;
        base[c] = bb;
    }
    __syncthreads();
    int W2 = 1;
    while (W2 < q && W2 < 32) W2 <<= 1;
    const int rpw = 32 / W2;
    const int grp = lane / W2, col = lane % W2;

    if (warp == 0 && CPL == 1 && q <= 16) {
        local_warp0_two_lane<MM>(m, q, bb, Es, Tb, tw, snap, snapw, deg, degl, sh, base, scale_g, nth, mp);
    } else if (warp == 0) {
        uint32_t scum[CPL];  // cumulative column scales over the chunk (Montgomery form)
#pragma unroll
        for (int k = 0; k < CPL; k++) scum[k] = mp.r1;
        for (int i = 0; i < bb; i++) {
            uint32_t *F = Tb + (i & 1) * tw;
            uint32_t *dg = F + mq;
            int *sn = snap + (i & 1) * snapw;
            int *s_sh = sn, *s_base = sn + q, *s_isp = sn + 2 * q, *s_pc = sn + 3 * q;
            // ---- elimination of order i
            uint32_t d[CPL][MM], tp[CPL][MM], sc[CPL];
            int rk[CPL];
#pragma unroll
            for (int k = 0; k < CPL; k++) {
                const int j = lane + 32 * k;
                const bool v = j < q;
                sc[k] = mp.r1;
                rk[k] = 1 << 20;
                if (v) {
                    int r0 = 0;
                    for (int c2 = 0; c2 < q; c2++)
                        r0 += (deg[c2] < deg[j] || (deg[c2] == deg[j] && c2 < j)) ? 1 : 0;
                    rk[k] = r0;
                    s_isp[j] = 0;
                    s_sh[j] = sh[j];
                    s_base[j] = base[j];
                }
                const uint32_t *er = Es + (size_t)(i - (v ? sh[j] : 0)) * mq + (v ? j : 0);
#pragma unroll
                for (int a2 = 0; a2 < MM; a2++) {
                    d[k][a2] = (v && a2 < m) ? to_mont(er[a2 * q], mp) : 0u;
                    tp[k][a2] = 0u;
                }
            }
            int np = 0;
            for (int step = 0; step < q; step++) {
                int mine = -1;
#pragma unroll
                for (int k = 0; k < CPL; k++)
                    if (rk[k] == step) mine = k;
                const unsigned who = __ballot_sync(0xffffffffu, mine >= 0);
                const int src = __ffs(who) - 1;
                int fr = -1;
                uint32_t sc_cur = 0;
                if (mine >= 0) {
#pragma unroll
                    for (int k = 0; k < CPL; k++)
                        if (k == mine) {
                            sc_cur = sc[k];
#pragma unroll
                            for (int a2 = MM - 1; a2 >= 0; a2--)
                                if (d[k][a2] != 0) fr = a2;
                        }
                }
                fr = __shfl_sync(0xffffffffu, fr, src);
                if (fr < 0) continue;
                const int jcur = __shfl_sync(0xffffffffu, lane + 32 * (mine >= 0 ? mine : 0), src);
                sc_cur = __shfl_sync(0xffffffffu, sc_cur, src);
                uint32_t pv[MM], pt[MM];
#pragma unroll
                for (int a2 = 0; a2 < MM; a2++) {
                    uint32_t x0 = 0, x1 = 0;
#pragma unroll
                    for (int k = 0; k < CPL; k++)
                        if (k == mine) { x0 = d[k][a2]; x1 = tp[k][a2]; }
                    pv[a2] = __shfl_sync(0xffffffffu, x0, src);
                    pt[a2] = __shfl_sync(0xffffffffu, x1, src);
                }
                uint32_t dc = 0;
#pragma unroll
                for (int a2 = 0; a2 < MM; a2++)
                    if (a2 == fr) dc = pv[a2];
                // col <- dc col - dj pivot: one Montgomery reduction of
                // dc*x + (p - dj)*y < 2 p^2 < p 2^32 per entry
#pragma unroll
                for (int k = 0; k < CPL; k++) {
                    if (rk[k] > step && rk[k] < (1 << 20)) {
                        uint32_t dj = 0;
#pragma unroll
                        for (int a2 = 0; a2 < MM; a2++)
                            if (a2 == fr) dj = d[k][a2];
                        if (dj != 0) {
                            const uint64_t ndj = mp.p - dj;
#pragma unroll
                            for (int a2 = 0; a2 < MM; a2++)
                                d[k][a2] = mont_redc((uint64_t)dc * d[k][a2] + ndj * pv[a2], mp);
#pragma unroll
                            for (int t = 0; t < MM; t++) {
                                if (t < np) tp[k][t] = mont_redc((uint64_t)dc * tp[k][t] + ndj * pt[t], mp);
                                else if (t == np) tp[k][t] = mont_redc(ndj * sc_cur, mp);
                            }
                            sc[k] = mont_mul(sc[k], dc, mp);
                        }
                    }
                }
                if (lane == 0) {
                    s_pc[np] = jcur;
                    s_isp[jcur] = 1;
                }
                np++;
            }
            __syncwarp();
            // publish the transform (normal form) and the local degree bounds
            int dln[CPL];
#pragma unroll
            for (int k = 0; k < CPL; k++) {
                const int j = lane + 32 * k;
                dln[k] = 0;
                if (j < q) {
                    int dl = degl[j];
#pragma unroll
                    for (int t = 0; t < MM; t++)
                        if (t < np) {
                            const uint32_t v = from_mont(tp[k][t], mp);
                            F[t * q + j] = v;
                            if (v) dl = max(dl, degl[s_pc[t]]);
                        }
                    dg[j] = from_mont(sc[k], mp);
                    scum[k] = mont_mul(scum[k], sc[k], mp);
                    dln[k] = dl;
                }
            }
            int dmx = 0;
#pragma unroll
            for (int k = 0; k < CPL; k++) dmx = max(dmx, dln[k]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) dmx = max(dmx, __shfl_xor_sync(0xffffffffu, dmx, off));
            if (lane == 0) {
                sn[3 * q + m] = np;
                sn[3 * q + m + 1] = dmx;
            }
            __syncwarp();
            named_arrive(BAR_T0 + (i & 1), nth);
            // ---- bookkeeping of order i: local degrees, pivots times x
#pragma unroll
            for (int k = 0; k < CPL; k++)
                if (lane + 32 * k < q) degl[lane + 32 * k] = dln[k];
            __syncwarp();
            for (int t = lane; t < np; t += 32) {
                const int c = s_pc[t];
                deg[c] += 1;
                degl[c] += 1;
                sh[c] += 1;
                base[c] -= 1;
            }
            __syncwarp();
            // ---- the next discrepancy (rows i, i+1) must be done
            named_sync(BAR_RR0 + (i & 1), nth);
        }
        // cumulative scales of this chunk into the running product
#pragma unroll
        for (int k = 0; k < CPL; k++) {
            const int j = lane + 32 * k;
            if (j < q) scale_g[j] = mont_mul(scale_g[j], scum[k], mp);
        }
    } else {
        // warps on warp 0's SM sub-partition (w % 4 == 0) take no rows, so
        // the elimination keeps its issue slots
        const bool worker = (warp & 3) != 0;
        const int ow = warp - 1 - (warp >> 2), nw = nwarps - nwarps / 4;
        const int NG = nw * rpw;        // row groups over all worker warps
        const int gg = ow * rpw + grp;  // this lane group's first row
        int jc[CPL];
        bool cok[CPL];
#pragma unroll
        for (int k = 0; k < CPL; k++) {
            jc[k] = CPL == 1 ? col : lane + 32 * k;
            cok[k] = jc[k] < q;
        }
        RowTransform<MM, CPL, KLAZY> tr;
        for (int i = 0; i < bb; i++) {
            named_sync(BAR_T0 + (i & 1), nth);
            const uint32_t *F = Tb + (i & 1) * tw;
            const uint32_t *dg = F + mq;
            const int *sn = snap + (i & 1) * snapw;
            const int *s_sh = sn, *s_base = sn + q, *s_isp = sn + 2 * q, *s_pc = sn + 3 * q;
            const int np = sn[3 * q + m], dl = sn[3 * q + m + 1];
            if (worker) tr.load(F, dg, s_pc, np, q, W2, grp, col, lane);
            int shc[CPL], bsc[CPL];
#pragma unroll
            for (int k = 0; k < CPL; k++) {
                shc[k] = cok[k] ? s_sh[jc[k]] : 0;
                bsc[k] = cok[k] ? s_base[jc[k]] : 0;
            }
            // window row (ip, a2) of column j sits at Es[((ip - sh[j]) m + a2) q + j]
            auto es = [&](bool ok, int ip, int a2, uint32_t *(&ptr)[CPL]) {
#pragma unroll
                for (int k = 0; k < CPL; k++)
                    ptr[k] = (ok && cok[k]) ? Es + ((size_t)(ip - shc[k]) * m + a2) * q + jc[k] : nullptr;
            };
            // rows i and i+1 first (the next discrepancy)
            if (worker) {
                const int r1 = (i + 1 < bb ? 2 : 1) * m;
                for (int row0 = ow * rpw; row0 < r1; row0 += NG) {
                    const int row = row0 + grp;
                    uint32_t *ptr[CPL];
                    es(row < r1, i + (row >= m ? 1 : 0), row - (row >= m ? m : 0), ptr);
                    tr.apply(ptr, mp);
                }
            }
            named_arrive(BAR_RR0 + (i & 1), nth);
            if (worker && np > 0) {
                // window orders i+2 .. bb-1: rows gg, gg + NG, ... walked incrementally
                const int wr = (bb - i - 2) > 0 ? (bb - i - 2) * m : 0;
                {
                    const int stepi = NG / m, stepa = NG - (NG / m) * m;
                    int ip = i + 2 + gg / m, a2 = gg - (gg / m) * m;
                    for (int row0 = ow * rpw; row0 < wr; row0 += NG) {
                        uint32_t *ptr[CPL];
                        es(row0 + grp < wr, ip, a2, ptr);
                        tr.apply(ptr, mp);
                        ip += stepi;
                        a2 += stepa;
                        if (a2 >= m) { a2 -= m; ip++; }
                    }
                }
                // Qtop rows; the next Qtop keeps the pivot columns of Qtop T
                for (int row0 = ow * rpw; row0 < m; row0 += NG) {
                    const int a2 = row0 + grp;
                    uint32_t *ptr[CPL];
#pragma unroll
                    for (int k = 0; k < CPL; k++) ptr[k] = (a2 < m && cok[k]) ? qt + a2 * q + jc[k] : nullptr;
                    tr.apply(ptr, mp);
#pragma unroll
                    for (int k = 0; k < CPL; k++)
                        if (ptr[k] && !s_isp[jc[k]]) *ptr[k] = 0;
                }
                // Ml coefficients 0..dl: rows (s2, x) walked incrementally
                {
                    const int mrows = (dl + 1) * q;
                    const int steps2 = NG / q, stepx = NG - (NG / q) * q;
                    int s2 = gg / q, x = gg - (gg / q) * q;
                    for (int row0 = ow * rpw; row0 < mrows; row0 += NG) {
                        const bool ok = row0 + grp < mrows;
                        uint32_t *ptr[CPL];
#pragma unroll
                        for (int k = 0; k < CPL; k++)
                            ptr[k] = (ok && cok[k]) ? Ml + ((size_t)(bsc[k] + s2) * q + x) * q + jc[k] : nullptr;
                        tr.apply(ptr, mp);
                        s2 += steps2;
                        x += stepx;
                        if (x >= q) { x -= q; s2++; }
                    }
                }
            }
            if (np == 0)  // no pivot: the next Qtop is zero
                for (int x = tid - 32; x < mq; x += nth - 32) qt[x] = 0;
        }
    }
    __syncthreads();
    for (int x = tid; x < (bb + 1) * qq; x += nth) {
        const int s2 = x / qq, c = x % q, y = (x / q) % q;
        Ml_g[x] = Ml[((size_t)(base[c] + s2) * q + y) * q + c];
    }
    for (int x = tid; x < mq; x += nth) qtop_g[x] = qt[x];
    for (int c = tid; c < q; c += nth) {
        deg_g[c] = deg[c];
        degl_g[c] = degl[c];
    }
    if (tid == 0) {
        // bound on the polynomial degree of the basis: column c's degree
        // minus the smallest starting degree (the row shifts)
        int dmx = 0;
        for (int c = 0; c < q; c++) dmx = max(dmx, deg[c] - dbase);
        *dmax_g = dmx;
    }
}

// ---- local M-Basis for wide blocks (q = m + n > 32; m <= 32, q <= 64): one
// block of LW_THREADS threads, every warp taking part in every phase of an
// order, with barriers between the phases.
//
//   ranks : the (degree, index) order of the columns, and the discrepancy
//           column registers: warp w holds columns w, w + 16, w + 32, w + 48,
//           lane a row a of each (and coefficient a of its transform);
//   elim  : one step per column in that order, ended once m pivots are found
//           (then every remaining column is zero on all m rows).  The owner
//           warp of the step's column finds its first nonzero row and, if
//           there is one, publishes the pivot column through a double-buffered
//           shared slot; after a barrier every warp reduces its later columns
//           by it, fraction-free as in k_local;
//   publish: the transform (normal form) and the local degree bounds;
//   rows  : every row of the window (orders i ..), of Qtop and of the chunk
//           transform Ml (coefficients 0 .. dl) times the transform, one row
//           per warp, the pivot residues read as shared-memory broadcasts;
//   shift : the pivot columns times x, moved in place: window orders i+1 ..
//           and Ml coefficients 1 .. dl+1 take the column's values one order /
//           one coefficient down, so that rows stay plain (no per-column
//           offsets).
// The pivots, the transforms, P and the degrees are those of k_local.
constexpr int LW_THREADS = 512;
constexpr int LW_WARPS = LW_THREADS / 32;
constexpr int LW_CPW = 64 / LW_WARPS;  // columns per warp in the elimination
constexpr int LW_SLOT = 68;            // pivot slot: 32 residues, 32 transform coefficients, fr, dc, scale

// dynamic shared memory of k_local_wide for chunks of b orders; the rows of
// the window and of the transform are padded to q + 1 words, so that a
// column (one residue per lane, rows apart) falls on distinct banks
__host__ __device__ constexpr size_t local_wide_bytes(int b, int m, int q) {
    return sizeof(uint32_t) * ((size_t)b * m * (q + 1) + (size_t)(b + 1) * q * q + (size_t)m * (q + 1) + (size_t)m * q +
                               64 + 2 * LW_SLOT) +
           sizeof(int) * (5 * 64 + 32 + 8);
}

template <int FOLDK>
__global__ void __launch_bounds__(LW_THREADS, 1)
    k_local_wide(int m, int n, int q, int bb, int nparts, const uint32_t *__restrict__ Epart,
                 uint32_t *__restrict__ qtop_g, int32_t *__restrict__ deg_g, uint32_t *__restrict__ Ml_g,
                 int32_t *__restrict__ degl_g, int *__restrict__ dmax_g, uint32_t *__restrict__ scale_g, int dbase,
                 ModP mp) {
    extern __shared__ uint32_t sm[];
    const int mq = m * q, qq = q * q, qs = q + 1;
    uint32_t *Es = sm;                            // [bb][m][qs]
    uint32_t *Ml = Es + (size_t)bb * m * qs;      // [bb+1][q][q]
    uint32_t *F = Ml + (size_t)(bb + 1) * qq;     // [m][qs] transform of the order
    uint32_t *qt = F + (size_t)m * qs;            // [m][q]
    uint32_t *dg = qt + mq;                       // [64]
    uint32_t *slot = dg + 64;                     // [2][LW_SLOT]
    int *deg = (int *)(slot + 2 * LW_SLOT);       // [64]
    int *degl = deg + 64;                         // [64] local degrees
    int *dln = degl + 64;                         // [64] local degrees after the transform
    int *colof = dln + 64;                        // [64] column of each rank
    int *isp = colof + 64;                        // [64] pivot flags of the order
    int *pcs = isp + 64;                          // [32] pivot columns in order
    int *misc = pcs + 32;                         // [0]: max local degree after the transform
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const uint32_t fc = mp.r1;  // 2^32 mod p
    (void)n;

    for (int x = tid; x < mq; x += LW_THREADS) qt[x] = qtop_g[x];
    __syncthreads();
    const int E = bb * mq;
    for (int x = tid; x < E; x += LW_THREADS) {
        unsigned long long v = 0;
        for (int b = 0; b < nparts; b++) v += Epart[(size_t)b * E + x];
        uint32_t e = red64(v, mp);
        if (x < mq) e = subm(e, qt[x], mp);
        Es[(x / q) * qs + x % q] = e;
    }
    for (int x = tid; x < (bb + 1) * qq; x += LW_THREADS) Ml[x] = (x < qq && x / q == x % q) ? 1u : 0u;
    for (int c = tid; c < 64; c += LW_THREADS) {
        deg[c] = c < q ? deg_g[c] : 0;
        degl[c] = 0;
    }
    uint32_t scum[LW_CPW];  // cumulative column scales over the chunk (Montgomery form)
#pragma unroll
    for (int k = 0; k < LW_CPW; k++) scum[k] = mp.r1;
    __syncthreads();

    for (int i = 0; i < bb; i++) {
        // ---- ranks and the discrepancy registers
        uint32_t d[LW_CPW], tp[LW_CPW], sc[LW_CPW];
        int rk[LW_CPW];
        {
            const int la = lane, lb = lane + 32;
            const int da = la < q ? deg[la] : 0, db = lb < q ? deg[lb] : 0;
#pragma unroll
            for (int k = 0; k < LW_CPW; k++) {
                const int c = warp + LW_WARPS * k;
                const bool cv = c < q;
                const int dc = cv ? deg[c] : 0;
                const bool xa = cv && la < q && (da < dc || (da == dc && la < c));
                const bool xb = cv && lb < q && (db < dc || (db == dc && lb < c));
                const int r = __popc(__ballot_sync(FULL, xa)) + __popc(__ballot_sync(FULL, xb));
                rk[k] = cv ? r : (1 << 20);
                d[k] = (cv && lane < m) ? to_mont(Es[((size_t)i * m + lane) * qs + c], mp) : 0u;
                tp[k] = 0u;
                sc[k] = mp.r1;
                if (cv && lane == 0) {
                    colof[r] = c;
                    isp[c] = 0;
                }
            }
        }
        if (tid == 0) misc[0] = 0;
        __syncthreads();
        // ---- elimination
        int np = 0;
        for (int step = 0; step < q && np < m; step++) {
            const int c = colof[step];
            uint32_t *sl = slot + (step & 1) * LW_SLOT;
            if ((c & (LW_WARPS - 1)) == warp) {
                const int kk = c / LW_WARPS;
                uint32_t v = 0, t = 0, s = 0;
#pragma unroll
                for (int k = 0; k < LW_CPW; k++)
                    if (k == kk) {
                        v = d[k];
                        t = tp[k];
                        s = sc[k];
                    }
                const int fr = __ffs(__ballot_sync(FULL, v != 0u)) - 1;
                if (fr >= 0) {
                    const uint32_t dcv = __shfl_sync(FULL, v, fr);
                    sl[lane] = v;
                    sl[32 + lane] = t;
                    if (lane == 0) {
                        sl[64] = (uint32_t)fr;
                        sl[65] = dcv;
                        sl[66] = s;
                        pcs[np] = c;
                        isp[c] = 1;
                    }
                } else if (lane == 0) {
                    sl[64] = 0xffffffffu;
                }
            }
            __syncthreads();
            const int fr = (int)sl[64];
            if (fr < 0) continue;
            const uint32_t pv = sl[lane], pt = sl[32 + lane], dcv = sl[65], scc = sl[66];
#pragma unroll
            for (int k = 0; k < LW_CPW; k++) {
                if (rk[k] > step && rk[k] < (1 << 20)) {
                    const uint32_t dj = __shfl_sync(FULL, d[k], fr);
                    if (dj != 0u) {
                        // col <- dc col - dj pivot: dc x + (p - dj) y < 2 p^2 < p 2^32
                        const uint32_t ndj = mp.p - dj;
                        d[k] = mont_redc(madw(ndj, pv, (unsigned long long)dcv * d[k]), mp);
                        if (lane < np) tp[k] = mont_redc(madw(ndj, pt, (unsigned long long)dcv * tp[k]), mp);
                        else if (lane == np) tp[k] = mont_redc((unsigned long long)ndj * scc, mp);
                        sc[k] = mont_mul(sc[k], dcv, mp);
                    }
                }
            }
            np++;
        }
        // ---- publish the transform (normal form) and the local degree bounds
#pragma unroll
        for (int k = 0; k < LW_CPW; k++) {
            const int c = warp + LW_WARPS * k;
            if (c < q) {
                const uint32_t fv = lane < np ? from_mont(tp[k], mp) : 0u;
                if (lane < np) F[lane * qs + c] = fv;
                const int v = __reduce_max_sync(FULL, fv != 0u ? degl[pcs[lane]] : 0);
                const int dl = max(degl[c], v);
                if (lane == 0) {
                    dg[c] = from_mont(sc[k], mp);
                    dln[c] = dl;
                    atomicMax(misc, dl);
                }
                scum[k] = mont_mul(scum[k], sc[k], mp);
            }
        }
        __syncthreads();
        const int dl = misc[0];
        // ---- rows times the transform
        if (np > 0) {
            const int ja = lane, jb = lane + 32;
            const bool vb = jb < q;
            uint32_t fa[32], fb[32];
#pragma unroll
            for (int t = 0; t < 32; t++) {
                fa[t] = t < np ? F[t * qs + ja] : 0u;
                fb[t] = (t < np && vb) ? F[t * qs + jb] : 0u;
            }
            const uint32_t ga = dg[ja], gb = vb ? dg[jb] : 0u;
            const int pcl = lane < np ? pcs[lane] : 0;  // lane t fetches the row's residue at pivot column t
            const int nwin = (bb - i) * m;
            const int nrows = nwin + m + (dl + 1) * q;
            for (int row = warp; row < nrows; row += LW_WARPS) {
                uint32_t *rp = row < nwin ? Es + ((size_t)i * m + row) * qs
                                          : (row < nwin + m ? qt + (row - nwin) * q : Ml + (size_t)(row - nwin - m) * q);
                const uint32_t xa = rp[ja], xb = vb ? rp[jb] : 0u, g = rp[pcl];
                // two accumulators per column (even and odd t), each folded
                // after FOLDK of its own products
                unsigned long long a0 = (unsigned long long)ga * xa, b0 = (unsigned long long)gb * xb;
                unsigned long long a1 = 0ull, b1 = 0ull;
#pragma unroll
                for (int t = 0; t < 32; t++) {
                    if (t < np) {
                        const uint32_t v = __shfl_sync(FULL, g, t);
                        if ((t & 1) == 0) {
                            a0 = madw(fa[t], v, a0);
                            b0 = madw(fb[t], v, b0);
                            if ((t / 2 + 2) % FOLDK == 0) {
                                a0 = fold2(a0, fc);
                                b0 = fold2(b0, fc);
                            }
                        } else {
                            a1 = madw(fa[t], v, a1);
                            b1 = madw(fb[t], v, b1);
                            if (((t + 1) / 2) % FOLDK == 0) {
                                a1 = fold2(a1, fc);
                                b1 = fold2(b1, fc);
                            }
                        }
                    }
                }
                // folded, each is below 2^62 + 2^32: their sum fits
                uint32_t ra = red64(fold2(a0, fc) + fold2(a1, fc), mp), rb = red64(fold2(b0, fc) + fold2(b1, fc), mp);
                if (row >= nwin && row < nwin + m) {  // the next Qtop keeps the pivot columns of Qtop T
                    if (!isp[ja]) ra = 0u;
                    if (vb && !isp[jb]) rb = 0u;
                }
                __syncwarp();
                rp[ja] = ra;
                if (vb) rp[jb] = rb;
                __syncwarp();
            }
        } else {
            for (int x = tid; x < mq; x += LW_THREADS) qt[x] = 0u;  // no pivot: the next Qtop is zero
        }
        __syncthreads();
        // ---- pivot columns times x (consecutive threads: the pivots of one
        // row, distinct columns)
        for (int w = tid; w < np * m; w += LW_THREADS) {
            const int a = w / np, c = pcs[w - a * np];
            for (int ip = bb - 1; ip > i; ip--)
                Es[((size_t)ip * m + a) * qs + c] = Es[((size_t)(ip - 1) * m + a) * qs + c];
        }
        for (int w = tid; w < np * q; w += LW_THREADS) {
            const int y = w / np, c = pcs[w - y * np];
            for (int s = dl + 1; s > 0; s--) Ml[((size_t)s * q + y) * q + c] = Ml[((size_t)(s - 1) * q + y) * q + c];
            Ml[(size_t)y * q + c] = 0u;
        }
        for (int c = tid; c < q; c += LW_THREADS) {
            degl[c] = dln[c] + isp[c];
            deg[c] += isp[c];
        }
        __syncthreads();
    }
    for (int x = tid; x < (bb + 1) * qq; x += LW_THREADS) Ml_g[x] = Ml[x];
    for (int x = tid; x < mq; x += LW_THREADS) qtop_g[x] = qt[x];
    for (int c = tid; c < q; c += LW_THREADS) {
        deg_g[c] = deg[c];
        degl_g[c] = degl[c];
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < LW_CPW; k++) {
            const int c = warp + LW_WARPS * k;
            if (c < q) scale_g[c] = mont_mul(scale_g[c], scum[k], mp);
        }
    }
    if (tid == 0) {
        // bound on the polynomial degree of the basis: column c's degree
        // minus the smallest starting degree (the row shifts)
        int dmx = 0;
        for (int c = 0; c < q; c++) dmx = max(dmx, deg[c] - dbase);
        *dmax_g = dmx;
    }
}

// P[t][r][c] /= S[c] (S in Montgomery form), t <= D
__global__ void k_unscale(uint32_t *__restrict__ P, int n, int q, int64_t D, const uint32_t *__restrict__ scale_g,
                          ModP mp) {
    __shared__ uint32_t inv[64];
    for (int c = threadIdx.x; c < q; c += blockDim.x) inv[c] = from_mont(mont_inv(scale_g[c], mp), mp);
    __syncthreads();
    const int64_t nq = (int64_t)n * q;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (D + 1) * nq; x += (int64_t)gridDim.x * blockDim.x)
        P[x] = mulm(P[x], inv[x % q], mp);
}

// ---- apply: P_new[t][r][c] = sum_{s <= degl[c]} sum_x P[t-s][r][x] Ml[s][x][c]
constexpr int APP_THREADS = 256;
constexpr int APP_TB = 8;  // coefficients per thread
constexpr int APP_CB = 4;  // columns per thread
static_assert(APP_TB == 8 && APP_CB == 4, "the register window and 16-byte loads assume an 8 x 4 tile");

// P' = P Ml (the chunk transform, logical layout: coefficient s of column c
// at Ml[s][.][c], zero above degl[c]), coefficients t0 .. t0 + TA - 1 of P' per
// block.  Coefficients above the new maximal column degree (*dmax_dev) are
// zero in P' and already zero in the target buffer (it held an older basis of
// no larger degree), so blocks beyond it return at once.  A thread owns a
// APP_TB x APP_CB tile (coefficients x columns) of one row r of P'.  For a
// fixed x it walks s: the P residues of step s+1 are those of step s shifted
// by one coefficient (circular register window, one new load per step), and
// the APP_CB residues of Ml are one 16-byte load (VEC).
template <int FOLDK, bool VEC>
__global__ void __launch_bounds__(APP_THREADS)
    k_apply(const uint32_t *__restrict__ P, uint32_t *__restrict__ Pn, int n, int q,
            const uint32_t *__restrict__ Ml_g, const int32_t *__restrict__ degl_g, int bb, int64_t Dbound,
            int TA, const int *__restrict__ dmax_dev, ModP mp) {
    extern __shared__ uint32_t sm[];
    uint32_t *Mls = sm;                               // (bb+1)*q*q
    uint32_t *Pss = Mls + (size_t)(bb + 1) * q * q;   // (TA + bb) * n * q
    __shared__ int degl[64];
    const int64_t dlim = min64(Dbound, (int64_t)*dmax_dev);
    const int64_t t0 = (int64_t)blockIdx.x * TA;
    if (t0 > dlim) return;
    const int ta = (int)min64(TA, dlim + 1 - t0);
    const int nq = n * q;
    const uint32_t fc = mp.r1;  // 2^32 mod p
    for (int x = threadIdx.x; x < (bb + 1) * q * q; x += APP_THREADS) Mls[x] = Ml_g[x];
    for (int x = threadIdx.x; x < q; x += APP_THREADS) degl[x] = degl_g[x];
    const int64_t pbase = t0 - bb;  // Pss[u] holds P[pbase + u]
    for (int x = threadIdx.x; x < (ta + bb) * nq; x += APP_THREADS) {
        const int64_t t = pbase + x / nq;
        Pss[x] = t >= 0 ? P[(size_t)t * nq + x % nq] : 0u;
    }
    __syncthreads();
    const int ntb = (ta + APP_TB - 1) / APP_TB, ncb = (q + APP_CB - 1) / APP_CB;
    for (int it = threadIdx.x; it < ntb * n * ncb; it += APP_THREADS) {
        const int cb = it % ncb, r = (it / ncb) % n, tb = it / (ncb * n);
        const int c0 = cb * APP_CB, tl0 = tb * APP_TB;
        bool cv[APP_CB];
        int smax = 0;
#pragma unroll
        for (int u = 0; u < APP_CB; u++) {
            cv[u] = c0 + u < q;
            if (cv[u]) smax = max(smax, degl[c0 + u]);
        }
        Acc2 acc[APP_TB][APP_CB];
#pragma unroll
        for (int k = 0; k < APP_TB; k++)
#pragma unroll
            for (int u = 0; u < APP_CB; u++) acc[k][u] = Acc2{0u, 0u};
        int cnt = 0;
        // coefficient t0 + tl0 + k - s of P is Pss row top - s + k
        const int top = tl0 + bb;
        for (int x = 0; x < q; x++) {
            const uint32_t *pc = Pss + r * q + x;          // row u at pc[u * nq]
            const uint32_t *mc = Mls + (size_t)x * q + c0;  // coefficient s at mc[s * q * q]
            uint32_t pw[APP_TB];                            // row top - s + k in slot (k - s) & 7
#pragma unroll
            for (int k = 0; k < APP_TB; k++) pw[k] = pc[(size_t)(top + k) * nq];
            for (int s0 = 0; s0 <= smax; s0 += 8) {
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int st = s0 + j;
                    if (st <= smax) {
                        if (st > 0) pw[(8 - j) & 7] = pc[(size_t)(top - st) * nq];
                        uint32_t mv[APP_CB];
                        ld4<VEC>(mc + (size_t)st * q * q, cv, mv);
#pragma unroll
                        for (int k = 0; k < APP_TB; k++)
#pragma unroll
                            for (int u = 0; u < APP_CB; u++) mac2(acc[k][u], pw[(k - j) & 7], mv[u]);
                        if (++cnt == FOLDK) {
#pragma unroll
                            for (int k = 0; k < APP_TB; k++)
#pragma unroll
                                for (int u = 0; u < APP_CB; u++) fold2w(acc[k][u], fc);
                            cnt = 0;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < APP_TB; k++) {
            const int tl = tl0 + k;
#pragma unroll
            for (int u = 0; u < APP_CB; u++)
                if (tl < ta && cv[u]) Pn[(size_t)(t0 + tl) * nq + r * q + c0 + u] = red64(acc2_u64(acc[k][u]), mp);
        }
    }
}

// Four consecutive residues through the read-only data cache (one 16-byte
// load when VEC), zero where the column is out of range.
template <bool VEC>
__device__ __forceinline__ void ldg4(const uint32_t *p, const bool (&cv)[4], uint32_t (&v)[4]) {
    if constexpr (VEC) {
        const uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = cv[u] ? __ldg(p + u) : 0u;
    }
}

// P' = P Ml for wide blocks (q > 32), where Ml and whole coefficients of P
// do not fit in shared memory together: block (coefficient tile of APW_TA,
// group of APW_RB rows of P); the tile's rows of P (with the bb coefficients
// below it) in shared memory, Ml through the read-only cache (it is shared by
// all blocks).  The thread tiles and the register window are those of k_apply.
constexpr int APW_RB = 4, APW_TA = 32;

__host__ __device__ constexpr size_t apply_wide_bytes(int b, int q) {
    return sizeof(uint32_t) * (size_t)(APW_TA + b) * APW_RB * q;
}

template <int FOLDK, bool VEC>
__global__ void __launch_bounds__(APP_THREADS, 2)
    k_apply_wide(const uint32_t *__restrict__ P, uint32_t *__restrict__ Pn, int n, int q,
                 const uint32_t *__restrict__ Ml_g, const int32_t *__restrict__ degl_g, int bb, int64_t Dbound,
                 const int *__restrict__ dmax_dev, ModP mp) {
    extern __shared__ uint32_t sm[];
    __shared__ int degl[64];
    const int64_t dlim = min64(Dbound, (int64_t)*dmax_dev);
    const int64_t t0 = (int64_t)blockIdx.x * APW_TA;
    if (t0 > dlim) return;
    const int ta = (int)min64(APW_TA, dlim + 1 - t0);
    const int r0 = blockIdx.y * APW_RB, rn = min(APW_RB, n - r0);
    const int nq = n * q, rq = APW_RB * q, qq = q * q;
    const uint32_t fc = mp.r1;  // 2^32 mod p
    for (int x = threadIdx.x; x < q; x += APP_THREADS) degl[x] = degl_g[x];
    const int64_t pbase = t0 - bb;  // sm[u rq + rl q + x] holds P[pbase + u][r0 + rl][x]
    for (int x = threadIdx.x; x < (ta + bb) * rq; x += APP_THREADS) {
        const int u = x / rq, rem = x - u * rq, rl = rem / q;
        const int64_t t = pbase + u;
        sm[x] = (t >= 0 && rl < rn) ? P[(size_t)t * nq + (size_t)(r0 + rl) * q + (rem - rl * q)] : 0u;
    }
    __syncthreads();
    const int ntb = (ta + APP_TB - 1) / APP_TB, ncb = (q + APP_CB - 1) / APP_CB;
    for (int it = threadIdx.x; it < ntb * APW_RB * ncb; it += APP_THREADS) {
        const int cb = it % ncb, rl = (it / ncb) % APW_RB, tb = it / (ncb * APW_RB);
        if (rl >= rn) continue;
        const int c0 = cb * APP_CB, tl0 = tb * APP_TB;
        bool cv[APP_CB];
        int smax = 0;
#pragma unroll
        for (int u = 0; u < APP_CB; u++) {
            cv[u] = c0 + u < q;
            if (cv[u]) smax = max(smax, degl[c0 + u]);
        }
        Acc2 acc[APP_TB][APP_CB];
#pragma unroll
        for (int k = 0; k < APP_TB; k++)
#pragma unroll
            for (int u = 0; u < APP_CB; u++) acc[k][u] = Acc2{0u, 0u};
        int cnt = 0;
        const int top = tl0 + bb;  // coefficient t0 + tl0 + k - s of P is slab row top - s + k
        for (int x = 0; x < q; x++) {
            const uint32_t *pc = sm + rl * q + x;       // slab row u at pc[u * rq]
            const uint32_t *mc = Ml_g + (size_t)x * q + c0;  // coefficient s at mc[s * qq]
            uint32_t pw[APP_TB];                        // slab row top - s + k in slot (k - s) & 7
#pragma unroll
            for (int k = 0; k < APP_TB; k++) pw[k] = pc[(size_t)(top + k) * rq];
            for (int s0 = 0; s0 <= smax; s0 += 8) {
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int st = s0 + j;
                    if (st <= smax) {
                        if (st > 0) pw[(8 - j) & 7] = pc[(size_t)(top - st) * rq];
                        uint32_t mv[APP_CB];
                        ldg4<VEC>(mc + (size_t)st * qq, cv, mv);
#pragma unroll
                        for (int k = 0; k < APP_TB; k++)
#pragma unroll
                            for (int u = 0; u < APP_CB; u++) mac2(acc[k][u], pw[(k - j) & 7], mv[u]);
                        if (++cnt == FOLDK) {
#pragma unroll
                            for (int k = 0; k < APP_TB; k++)
#pragma unroll
                                for (int u = 0; u < APP_CB; u++) fold2w(acc[k][u], fc);
                            cnt = 0;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < APP_TB; k++) {
            const int tl = tl0 + k;
#pragma unroll
            for (int u = 0; u < APP_CB; u++)
                if (tl < ta && cv[u])
                    Pn[(size_t)(t0 + tl) * nq + (size_t)(r0 + rl) * q + c0 + u] = red64(acc2_u64(acc[k][u]), mp);
        }
    }
}

// ---------------------------------------------------------------- readout

// choose the n columns of least (degree, index)
__global__ void k_select(const int32_t *__restrict__ deg, int q, int n, int32_t *__restrict__ sel,
                         int32_t *__restrict__ delta) {
    int c = threadIdx.x;
    if (c >= q) return;
    int rk = 0;
    for (int c2 = 0; c2 < q; c2++) rk += (deg[c2] < deg[c] || (deg[c2] == deg[c] && c2 < c)) ? 1 : 0;
    if (rk < n) {
        sel[rk] = c;
        delta[rk] = deg[c];
    }
}

// G[t][r][j] for t < T: reversed (F) or plain (P) coefficients of the selected columns
__global__ void k_extract(const uint32_t *__restrict__ P, int n, int q, const int32_t *__restrict__ sel,
                          const int32_t *__restrict__ delta, int64_t T, int reversed, int64_t Dcap,
                          uint32_t *__restrict__ G) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T * n * n) return;
    const int64_t t = i / (n * n);
    const int r = (int)((i / n) % n), j = (int)(i % n);
    const int64_t dj = delta[j];
    int64_t src = reversed ? dj - t : t;
    uint32_t v = 0;
    if (src >= 0 && src <= dj && src <= Dcap) v = P[((size_t)src * n + r) * q + sel[j]];
    G[i] = v;
}

// x-adic valuation of det G over F_p[[x]] / x^T: g laid out [(i*n + j)*T + t].
constexpr int VAL_THREADS = 256;

__global__ void __launch_bounds__(VAL_THREADS)
    k_valuation(const uint32_t *__restrict__ G, uint32_t *__restrict__ g, int n, int T,
                int64_t *__restrict__ out, ModP mp) {
    extern __shared__ uint32_t sm[];
    uint32_t *inv = sm;              // T
    uint32_t *mu = inv + T;          // n * T
    int *rdone = (int *)(mu + (size_t)n * T);
    int *cdone = rdone + n;
    __shared__ unsigned long long best;
    const int tid = threadIdx.x;
    for (int64_t i = tid; i < (int64_t)n * n * T; i += blockDim.x) {
        int64_t t = i % T, ij = i / T;
        g[i] = G[(size_t)t * n * n + ij];
    }
    for (int i = tid; i < n; i += blockDim.x) rdone[i] = cdone[i] = 0;
    __syncthreads();
    int prec = T;
    int64_t total = 0;
    for (int step = 0; step < n; step++) {
        if (tid == 0) best = ~0ull;
        __syncthreads();
        // pivot: least valuation, then least (row, col)
        for (int ij = tid; ij < n * n; ij += blockDim.x) {
            const int i = ij / n, j = ij % n;
            if (rdone[i] || cdone[j]) continue;
            const uint32_t *e = g + (size_t)ij * T;
            for (int t = 0; t < prec; t++)
                if (e[t]) {
                    unsigned long long key = ((unsigned long long)t << 40) | ((unsigned long long)i << 20) | j;
                    atomicMin(&best, key);
                    break;
                }
        }
        __syncthreads();
        const unsigned long long key = best;
        if (key == ~0ull) {
            if (tid == 0) *out = -1;
            return;
        }
        const int bv = (int)(key >> 40), bi = (int)((key >> 20) & 0xFFFFF), bj = (int)(key & 0xFFFFF);
        total += bv;
        const int np_ = prec - bv;
        const uint32_t *piv = g + ((size_t)bi * n + bj) * T + bv;  // unit part u
        if (tid == 0) {
            inv[0] = invm(piv[0], mp);
            for (int t = 1; t < np_; t++) {
                unsigned long long acc = 0;
                for (int s = 1; s <= t; s++) acc = red64(acc + (unsigned long long)piv[s] * inv[t - s], mp);
                inv[t] = mulm(subm(0, (uint32_t)acc, mp), inv[0], mp);
            }
        }
        __syncthreads();
        // mu_i = (g[i][bj] / x^bv) * inv  mod x^np_
        for (int w = tid; w < n * np_; w += blockDim.x) {
            const int i = w / np_, t = w % np_;
            if (rdone[i] || i == bi) continue;
            const uint32_t *gi = g + ((size_t)i * n + bj) * T + bv;
            unsigned long long acc = 0;
            for (int s = 0; s <= t; s++) acc = red64(acc + (unsigned long long)gi[s] * inv[t - s], mp);
            mu[(size_t)i * T + t] = (uint32_t)acc;
        }
        __syncthreads();
        // g[i][j] -= mu_i * g[bi][j]  mod x^np_, zero beyond
        for (int w = tid; w < n * n; w += blockDim.x) {
            const int i = w / n, j = w % n;
            if (rdone[i] || i == bi || cdone[j]) continue;
            uint32_t *gij = g + (size_t)w * T;
            const uint32_t *gb = g + ((size_t)bi * n + j) * T;
            const uint32_t *mi = mu + (size_t)i * T;
            for (int t = np_ - 1; t >= 0; t--) {
                unsigned long long acc = 0;
                for (int s = 0; s <= t; s++) acc = red64(acc + (unsigned long long)mi[s] * gb[t - s], mp);
                gij[t] = subm(gij[t], (uint32_t)acc, mp);
            }
            for (int t = np_; t < T; t++) gij[t] = 0;
        }
        __syncthreads();
        if (tid == 0) {
            rdone[bi] = 1;
            cdone[bj] = 1;
        }
        prec = np_;
        __syncthreads();
    }
    if (tid == 0) *out = total;
}

}  // namespace

// Blocked M-Basis over L orders.  [S | -I_m] (d_deg_in == nullptr): S holds
// L x m x n, d_P receives the first nr = n rows of the basis, d_deg the
// shifted degrees.  A general residual F (d_deg_in given): S holds L x m x q,
// nr = q, the basis starts at I_q with the degrees d_deg_in, and dbase is
// their minimum.  *dmax_out (optional): a bound on the basis's polynomial
// degree.
static wr_status mbasis_run(wr_ctx *ctx, const uint32_t *d_S, int64_t L, int m, int nr, int n, uint32_t p,
                            uint32_t *d_P, int32_t *d_deg, const int32_t *d_deg_in, int dbase, int64_t Dcap,
                            int64_t *dmax_out) {
    const int q = m + n;
    const ModP mp = make_modp(p);
    cudaStream_t s = ctx->stream;
    const size_t nq = (size_t)nr * q;
    WR_CUDA(cudaMemsetAsync(d_P, 0, sizeof(uint32_t) * (Dcap + 1) * nq, s));
    DevBuf P2, qtop, dmax, Epart, Ml, degl, scale;
    WR_TRY(dev_alloc(ctx, P2, sizeof(uint32_t) * (Dcap + 1) * nq));
    WR_CUDA(cudaMemsetAsync(P2.ptr, 0, P2.bytes, s));
    WR_TRY(dev_alloc(ctx, qtop, sizeof(uint32_t) * m * q));
    WR_TRY(dev_alloc(ctx, dmax, sizeof(int)));
    k_init_basis<<<1, 256, 0, s>>>(d_P, nr, n, q, d_deg, d_deg_in, qtop.as<uint32_t>(), m, dmax.as<int>());
    WR_LAUNCHED(ctx);

    // chunk size b and tiles: every kernel's shared memory must fit
    const size_t budget = std::min<size_t>(ctx->smem_optin, 227 * 1024) - 1024;
    auto local_bytes = [&](int b) {
        return sizeof(uint32_t) * ((size_t)b * m * q + (size_t)(2 * b + 1) * q * q + 3 * (size_t)m * q + 2 * q) +
               sizeof(int) * (4 * q + 2 * (3 * q + m + 2));
    };
    auto window_bytes = [&](int TT, int b) {
        const int nib = (b + WIN_IB - 1) / WIN_IB;
        return sizeof(uint32_t) * ((size_t)TT * nq + (size_t)(nib * WIN_IB + TT - 1) * m * nr);
    };
    auto apply_bytes = [&](int ta, int b) { return sizeof(uint32_t) * ((size_t)(b + 1) * q * q + (size_t)(ta + b) * nq); };
    // wide blocks (q > 32): k_local_wide and k_apply_wide, and chunks one
    // order shorter at a time (their shared memory grows in steps of a few KB)
    const bool wide = q > 32;
    auto local_need = [&](int b) { return wide ? local_wide_bytes(b, m, q) : local_bytes(b); };
    auto apply_need = [&](int ta, int b) { return wide ? apply_wide_bytes(b, q) : apply_bytes(ta, b); };
    int bmax = ctx->sigma_chunk > 0 ? std::min(ctx->sigma_chunk, 64) : (wide ? SIGMA_CHUNK_WIDE : SIGMA_CHUNK_DEFAULT),
        TT = 32, TA = 64;
    for (;;) {
        while (TT > 4 && window_bytes(TT, bmax) > budget) TT /= 2;
        while (TA > APP_TB && apply_need(TA, bmax) > budget) TA /= 2;
        if (local_need(bmax) <= budget && window_bytes(TT, bmax) <= budget && apply_need(TA, bmax) <= budget) break;
        if (bmax == 1) return fail(WR_EINVAL, "block sizes too large for shared memory");
        bmax = wide ? bmax - 1 : bmax / 2;
        TT = 32;
        TA = 64;
    }
    if (wide) TA = APW_TA;
    const int nparts_max = std::max(1, 2 * ctx->num_sms);
    WR_TRY(dev_alloc(ctx, Epart, sizeof(uint32_t) * (size_t)nparts_max * bmax * m * q));
    WR_TRY(dev_alloc(ctx, Ml, sizeof(uint32_t) * (size_t)(bmax + 1) * q * q));
    WR_TRY(dev_alloc(ctx, degl, sizeof(int32_t) * q));
    WR_TRY(dev_alloc(ctx, scale, sizeof(uint32_t) * q));
    {
        std::vector<uint32_t> one(q, mp.r1);  // Montgomery form of 1
        WR_CUDA(cudaMemcpyAsync(scale.ptr, one.data(), sizeof(uint32_t) * q, cudaMemcpyHostToDevice, s));
        WR_CUDA(cudaStreamSynchronize(s));
    }
    const bool lazy16 = mp.lazy >= 16;
    const bool vec = q % 4 == 0;
    // fold interval of the lazily reduced sums: 14 (p < 2^30), 3 (2^32 mod p
    // small, as for p = 2^31 - 19), else 2
    const int fk = fold_products(p), fold = fk >= 14 ? 14 : (fk >= 3 ? 3 : 2);
    // order tiles of 4 for chunks of at most 4 orders (8 would idle half the tile)
    auto win_for = [&](int b) {
        if (b <= 4)
            return fold == 14 ? (vec ? k_window<14, true, 4> : k_window<14, false, 4>)
                   : fold == 3 ? (vec ? k_window<3, true, 4> : k_window<3, false, 4>)
                               : (vec ? k_window<2, true, 4> : k_window<2, false, 4>);
        return fold == 14 ? (vec ? k_window<14, true, 8> : k_window<14, false, 8>)
               : fold == 3 ? (vec ? k_window<3, true, 8> : k_window<3, false, 8>)
                           : (vec ? k_window<2, true, 8> : k_window<2, false, 8>);
    };
    auto *kwin = win_for(bmax);
    auto *kwin_tail = win_for(std::min<int64_t>(bmax, L % bmax ? L % bmax : bmax));
    auto *kapp = fold == 14 ? (vec ? k_apply<14, true> : k_apply<14, false>)
                 : fold == 3 ? (vec ? k_apply<3, true> : k_apply<3, false>)
                             : (vec ? k_apply<2, true> : k_apply<2, false>);
    auto *kapp_w = fold == 14 ? (vec ? k_apply_wide<14, true> : k_apply_wide<14, false>)
                   : fold == 3 ? (vec ? k_apply_wide<3, true> : k_apply_wide<3, false>)
                               : (vec ? k_apply_wide<2, true> : k_apply_wide<2, false>);
    DevBuf Esum;
    WR_TRY(dev_alloc(ctx, Esum, sizeof(uint32_t) * (size_t)bmax * m * q));
    using LocalFn = void (*)(int, int, int, int, int, const uint32_t *, uint32_t *, int32_t *, uint32_t *, int32_t *,
                             int *, uint32_t *, int, ModP);
    LocalFn kloc;
    if (wide)
        kloc = fold == 14 ? k_local_wide<14> : (fold == 3 ? k_local_wide<3> : k_local_wide<2>);
    else if (m <= 8)
        kloc = lazy16 ? k_local<8, 1, 16> : k_local<8, 1, 4>;
    else
        kloc = lazy16 ? k_local<32, 1, 16> : k_local<32, 1, 4>;
    WR_CUDA(cudaFuncSetAttribute(kwin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));
    WR_CUDA(cudaFuncSetAttribute(kwin_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));
    WR_CUDA(cudaFuncSetAttribute(kloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));
    WR_CUDA(cudaFuncSetAttribute(kapp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));
    WR_CUDA(cudaFuncSetAttribute(kapp_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));

    uint32_t *Pcur = d_P, *Pnext = P2.as<uint32_t>();
    int64_t Dbound = 1;
    // early termination on a sequence in flight: a quiet-order count per
    // chunk in host-mapped memory; the loop stays ET_LAG chunks ahead of the
    // device and stops once ctx->early_term consecutive orders were quiet
    SeqFeed *feed = d_deg_in ? nullptr : ctx->feed;
    const bool early = feed && ctx->early_term > 0;
    constexpr int ET_RING = 8, ET_LAG = 2;
    long long *et_host = nullptr, *et_host_dev = nullptr;
    cudaEvent_t et_ev[ET_RING] = {};
    DevBuf et_count;
    struct EtCleanup {
        long long *&h;
        cudaEvent_t *ev;
        ~EtCleanup() {
            if (h) cudaFreeHost(h);
            for (int i = 0; i < ET_RING; i++)
                if (ev[i]) cudaEventDestroy(ev[i]);
        }
    } et_cleanup{et_host, et_ev};
    if (early) {
        WR_CUDA(cudaHostAlloc((void **)&et_host, sizeof(long long) * ET_RING, cudaHostAllocMapped));
        for (int i = 0; i < ET_RING; i++) et_host[i] = -1;
        WR_CUDA(cudaHostGetDevicePointer((void **)&et_host_dev, et_host, 0));
        for (int i = 0; i < ET_RING; i++) WR_CUDA(cudaEventCreateWithFlags(&et_ev[i], WAIT_EVENT_FLAGS));
        WR_TRY(dev_alloc(ctx, et_count, sizeof(long long)));
        WR_CUDA(cudaMemsetAsync(et_count.ptr, 0, sizeof(long long), s));
    }
    int64_t Lused = L;
    // profiling: events around the three kernels of every 16th chunk
    cudaEvent_t pe[4] = {nullptr, nullptr, nullptr, nullptr};
    double pw = 0, pl = 0, pa = 0;
    int64_t nchunks = (L + bmax - 1) / bmax, sampled = 0;  // (profiling extrapolates to all L orders)
    if (ctx->profiling)
        for (auto &e : pe) WR_CUDA(cudaEventCreate(&e));
    for (int64_t k0 = 0; k0 < L; k0 += bmax) {
        const int bb = (int)std::min<int64_t>(bmax, L - k0);
        const bool prof = ctx->profiling && ((k0 / bmax) % 16 == 0);
        const int64_t chunk = k0 / bmax;
        if (early && chunk >= ET_LAG) {
            const int slot = (int)((chunk - ET_LAG) % ET_RING);
            WR_CUDA(cudaEventSynchronize(et_ev[slot]));
            if (*(volatile long long *)(et_host + slot) >= ctx->early_term) {
                Lused = k0;  // the generator is stable: the chunks so far are the whole basis
                feed->stop_at.store(k0);
                break;
            }
        }
        // a sequence still in flight: the window reads S rows below k0 + bb
        // rounded up to its order tile
        if (feed) WR_TRY(feed_wait(ctx, feed, std::min<int64_t>(L, k0 + (bb + WIN_IB - 1) / WIN_IB * WIN_IB)));
        if (prof) WR_CUDA(cudaEventRecord(pe[0], s));
        // window: split coefficients [0, min(Dbound, k0 + bb - 1)] over the blocks
        const int64_t tspan = std::min<int64_t>(Dbound, k0 + bb - 1) + 1;
        const int nparts = (int)std::min<int64_t>(nparts_max, std::max<int64_t>(1, (tspan + TT - 1) / TT));
        const int64_t tper = (tspan + nparts - 1) / nparts;
        (bb == bmax ? kwin : kwin_tail)<<<nparts, WIN_THREADS, window_bytes(TT, bb), s>>>(d_S, L, m, nr, q, Pcur, k0, bb, TT, tper,
                                                                dmax.as<int>(), Epart.as<uint32_t>(), mp);
        WR_LAUNCHED(ctx);
        const uint32_t *Ewin = Epart.as<uint32_t>();
        if (nparts > 1) {
            const int64_t E = (int64_t)bb * m * q;
            k_sum_parts<<<(unsigned)((E + 31) / 32), 256, 0, s>>>(nparts, E, Epart.as<uint32_t>(),
                                                                  Esum.as<uint32_t>(), mp);
            WR_LAUNCHED(ctx);
            Ewin = Esum.as<uint32_t>();
        }
        if (early) {
            k_quiet<<<1, 64, 0, s>>>(Ewin, bb, m, n, q, d_deg, k0, et_count.as<long long>(),
                                     et_host_dev + chunk % ET_RING);
            WR_LAUNCHED(ctx);
        }
        if (prof) WR_CUDA(cudaEventRecord(pe[1], s));
        kloc<<<1, wide ? LW_THREADS : local_threads(m <= 8 ? 8 : 32, 1), local_need(bb), s>>>(
            m, n, q, bb, 1, Ewin, qtop.as<uint32_t>(), d_deg, Ml.as<uint32_t>(),
            degl.as<int32_t>(), dmax.as<int>(), scale.as<uint32_t>(), dbase, mp);
        WR_LAUNCHED(ctx);
        if (prof) WR_CUDA(cudaEventRecord(pe[2], s));
        if (Dbound + bb > Dcap + 1) return fail(WR_EINVAL, "sigma-basis degree cap too small");
        const int64_t Dnew = std::min<int64_t>(Dbound + bb, Dcap);
        if (wide)
            kapp_w<<<dim3((unsigned)((Dnew + TA) / TA), (unsigned)((nr + APW_RB - 1) / APW_RB)), APP_THREADS,
                     apply_need(TA, bb), s>>>(Pcur, Pnext, nr, q, Ml.as<uint32_t>(), degl.as<int32_t>(), bb, Dnew,
                                              dmax.as<int>(), mp);
        else
            kapp<<<(unsigned)((Dnew + TA) / TA), APP_THREADS, apply_bytes(TA, bb), s>>>(
                Pcur, Pnext, nr, q, Ml.as<uint32_t>(), degl.as<int32_t>(), bb, Dnew, TA, dmax.as<int>(), mp);
        WR_LAUNCHED(ctx);
        if (prof) {
            WR_CUDA(cudaEventRecord(pe[3], s));
            WR_CUDA(cudaEventSynchronize(pe[3]));
            float a = 0, b = 0, c = 0;
            cudaEventElapsedTime(&a, pe[0], pe[1]);
            cudaEventElapsedTime(&b, pe[1], pe[2]);
            cudaEventElapsedTime(&c, pe[2], pe[3]);
            pw += a;
            pl += b;
            pa += c;
            sampled++;
        }
        if (early) WR_CUDA(cudaEventRecord(et_ev[chunk % ET_RING], s));
        std::swap(Pcur, Pnext);
        Dbound = Dnew;
    }
    if (feed) feed->orders_used = Lused;
    if (ctx->profiling) {
        for (auto &e : pe) cudaEventDestroy(e);
        const double scale = sampled ? (double)nchunks / sampled : 0.0;  // extrapolate the samples
        ctx->last.sigma_window_ms += pw * scale;
        ctx->last.sigma_local_ms += pl * scale;
        ctx->last.sigma_apply_ms += pa * scale;
    }
    if (Pcur != d_P)
        WR_CUDA(cudaMemcpyAsync(d_P, Pcur, sizeof(uint32_t) * (Dbound + 1) * nq, cudaMemcpyDeviceToDevice, s));
    // divide the cumulative column scales out of P
    k_unscale<<<(unsigned)std::min<int64_t>(((Dbound + 1) * nq + 255) / 256, (int64_t)ctx->num_sms * 8), 256, 0, s>>>(
        d_P, nr, q, Dbound, scale.as<uint32_t>(), mp);
    WR_LAUNCHED(ctx);
    if (dmax_out) {
        int h = 0;
        WR_CUDA(cudaMemcpyAsync(&h, dmax.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        WR_CUDA(sync_stream_blocking(s));
        *dmax_out = std::min<int64_t>(std::max(h, 0), Dbound);
    }
    WR_CUDA(sync_stream_blocking(s));  // (trailing a sequence: as long as the sequence)
    return WR_OK;
}

// F = [S | -I_m]: coefficients [k0, k1) of the L x m x q residual of the whole problem
__global__ void k_build_F(const uint32_t *__restrict__ S, int64_t k0, int64_t k1, int m, int n, uint32_t p,
                          uint32_t *__restrict__ F) {
    const int q = m + n;
    const int64_t total = (k1 - k0) * m * q;
    for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < total; y += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = y + k0 * m * q;
        const int64_t k = x / (m * q);
        const int rem = (int)(x - k * m * q), a = rem / q, c = rem % q;
        F[x] = c < n ? S[((size_t)k * m + a) * n + c] : ((k == 0 && c - n == a) ? p - 1 : 0u);
    }
}

// P[t][r][c] = M[t][r][c] for the first n of the q rows, t <= D
__global__ void k_top_rows(const uint32_t *__restrict__ M, int64_t D, int n, int q, uint32_t *__restrict__ P) {
    const int64_t total = (D + 1) * n * q;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = x / ((int64_t)n * q);
        const int rem = (int)(x - t * n * q);
        P[x] = M[((size_t)t * q + rem / q) * q + rem % q];
    }
}

// PM-Basis (Section 2.4): the sigma-basis of the residual F (d orders, m x q)
// for the starting degrees in d_deg (updated to the final degrees) is M1 M2,
// M1 the basis of the first h orders and M2 that of the residual
// R = (F M1) div x^h mod x^(d-h), the latter started from M1's degrees.  The
// leaves (d <= leaf) run the blocked M-Basis on a general residual; the
// residual and the product are polynomial matrix products by NTT (CRT over
// three FFT primes).  Each leaf's basis is the order-by-order one, so M is.
static wr_status pm_basis_rec(wr_ctx *ctx, const uint32_t *F, int64_t d, int m, int q, uint32_t p,
                              int32_t *d_deg, int64_t leaf, DevBuf &M, int64_t &DM) {
    cudaStream_t s = ctx->stream;
    std::vector<int32_t> h0(q);
    WR_CUDA(cudaMemcpyAsync(h0.data(), d_deg, sizeof(int32_t) * q, cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    const int dbase = *std::min_element(h0.begin(), h0.end());
    if (d <= leaf) {
        WR_TRY(dev_alloc(ctx, M, sizeof(uint32_t) * (size_t)(d + 2) * q * q));
        DevBuf degin;
        WR_TRY(dev_alloc(ctx, degin, sizeof(int32_t) * q));
        WR_CUDA(cudaMemcpyAsync(degin.ptr, d_deg, sizeof(int32_t) * q, cudaMemcpyDeviceToDevice, s));
        return mbasis_run(ctx, F, d, m, q, q - m, p, M.as<uint32_t>(), d_deg, degin.as<int32_t>(), dbase, d + 1, &DM);
    }
    int64_t h = ((d / 2 + 63) / 64) * 64;
    if (h >= d) h = d / 2;
    DevBuf M1, M2, R;
    int64_t DM1 = 0, DM2 = 0;
    WR_TRY(pm_basis_rec(ctx, F, h, m, q, p, d_deg, leaf, M1, DM1));
    WR_TRY(dev_alloc(ctx, R, sizeof(uint32_t) * (size_t)(d - h) * m * q));
    WR_TRY(polymat_mul(ctx, F, d, M1.as<uint32_t>(), DM1 + 1, m, q, q, h, d, p, R.as<uint32_t>()));
    WR_TRY(pm_basis_rec(ctx, R.as<uint32_t>(), d - h, m, q, p, d_deg, leaf, M2, DM2));
    R.release();
    // degree of M: at most DM1 + DM2, and at most the largest final degree
    // minus the smallest starting one
    std::vector<int32_t> h1(q);
    WR_CUDA(cudaMemcpyAsync(h1.data(), d_deg, sizeof(int32_t) * q, cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    const int64_t bound = (int64_t)*std::max_element(h1.begin(), h1.end()) - dbase;
    DM = std::max<int64_t>(0, std::min<int64_t>(DM1 + DM2, bound));
    WR_TRY(dev_alloc(ctx, M, sizeof(uint32_t) * (size_t)(DM + 2) * q * q));
    WR_CUDA(cudaMemsetAsync(M.ptr, 0, M.bytes, s));
    return polymat_mul(ctx, M1.as<uint32_t>(), DM1 + 1, M2.as<uint32_t>(), DM2 + 1, q, q, q, 0, DM + 1, p,
                       M.as<uint32_t>());
}

static int64_t sigma_leaf_for(const wr_ctx *ctx, int m, int n) {
    return ctx->sigma_leaf > 0 ? ctx->sigma_leaf : (m + n > 32 ? SIGMA_LEAF_WIDE : SIGMA_LEAF_DEFAULT);
}

// PM-Basis (else the blocked M-Basis) for L orders; early termination needs
// the order-by-order basis (PM-Basis splits the orders in halves and so needs
// all of them from the start)
bool sigma_uses_pm(const wr_ctx *ctx, int64_t L, int m, int n, bool early) {
    const int64_t leaf = sigma_leaf_for(ctx, m, n);
    const bool automatic = ctx->sigma_leaf <= 0;
    return !(early || L <= leaf || (automatic && L <= (m + n > 32 ? SIGMA_PM_MIN_L_WIDE : SIGMA_PM_MIN_L)));
}

bool sigma_pm_trailing(const wr_ctx *ctx, int64_t L, int m, int n) {
    return sigma_uses_pm(ctx, L, m, n, ctx->early_term > 0) && L > 2 * sigma_leaf_for(ctx, m, n);
}

wr_status sigma_basis(wr_ctx *ctx, const uint32_t *d_S, int64_t L, int m, int n, uint32_t p,
                      uint32_t *d_P, int32_t *d_deg, int64_t Dcap) {
    if (m < 1 || n < 1 || m > 32 || n > 32) return fail(WR_EINVAL, "block sizes must be in 1..32");
    ctx->last.sigma_window_ms = ctx->last.sigma_local_ms = ctx->last.sigma_apply_ms = 0.0;
    ctx->last.sigma_product_ms = 0.0;
    const int64_t leaf = sigma_leaf_for(ctx, m, n);
    const bool early = ctx->feed && ctx->early_term > 0;
    if (!sigma_uses_pm(ctx, L, m, n, early))
        return mbasis_run(ctx, d_S, L, m, n, n, p, d_P, d_deg, nullptr, 0, Dcap, nullptr);
    const int q = m + n;
    cudaStream_t s = ctx->stream;
    DevBuf F, M;
    WR_TRY(dev_alloc(ctx, F, sizeof(uint32_t) * (size_t)L * m * q));
    auto build_F = [&](int64_t k0, int64_t k1) -> wr_status {
        if (k1 <= k0) return WR_OK;
        const unsigned g = (unsigned)std::min<int64_t>(((k1 - k0) * m * q + 255) / 256, (int64_t)ctx->num_sms * 16);
        k_build_F<<<g, 256, 0, s>>>(d_S, k0, k1, m, n, p, F.as<uint32_t>());
        WR_LAUNCHED(ctx);
        return WR_OK;
    };
    std::vector<int32_t> deg0(q);
    for (int c = 0; c < q; c++) deg0[c] = c < n ? 0 : 1;
    WR_CUDA(cudaMemcpyAsync(d_deg, deg0.data(), sizeof(int32_t) * q, cudaMemcpyHostToDevice, s));
    WR_CUDA(cudaStreamSynchronize(s));
    int64_t DM = 0;
    // Trailing a sequence still in flight: the orders are taken in segments
    // [h_{k-1}, h_k) as the sequence publishes them.  A segment's residual is
    // R_k = (F M) div x^h_{k-1} mod x^(h_k - h_{k-1}) (a middle product of F's
    // coefficients [h_{k-1} - deg M, h_k) and the basis M of the orders before
    // it), its sigma-basis M_k starts from M's degrees, and M <- M M_k:
    // PM-Basis's split at h_{k-1}, applied once per segment.  Each segment is
    // about half of the orders still to come but at most a quarter of all
    // (the first starts when a quarter of the terms are in), down to two
    // leaves, so that what is left after the sequence's last term is one short
    // segment and two products.  (Segments that take every term finished meanwhile, from the
    // first sixteenth on, were measured slower on the 1.9M x 1.95M block-32
    // matrix: their kernels ran beside the SpMM for the whole sequence, each
    // segment with its two products, and cost the SpMM more than the shorter
    // tail saved.)
    if (ctx->feed && L > 2 * leaf) {
        const int64_t seg_min = 2 * leaf;
        std::vector<int32_t> hd(q);
        int64_t hprev = 0;
        for (int k = 0; hprev < L; k++) {
            const int64_t rem = L - hprev;
            const int64_t half = std::min<int64_t>(rem / 2, L / 4);
            const int64_t hk =
                hprev + (rem <= 2 * seg_min ? rem : std::max<int64_t>(seg_min, ((half + 63) / 64) * 64));
            const int64_t d = hk - hprev;
            WR_TRY(feed_wait(ctx, ctx->feed, hk));
            WR_TRY(build_F(hprev, hk));
            DevBuf R, Mk;
            int64_t DMk = 0;
            if (k > 0) {
                // R_i = sum_j F_j M_{i-j}, j in [i - DM, i]: F from hprev - DM on
                const int64_t off = std::max<int64_t>(0, hprev - DM);
                WR_TRY(dev_alloc(ctx, R, sizeof(uint32_t) * (size_t)d * m * q));
                WR_TRY(polymat_mul(ctx, F.as<uint32_t>() + (size_t)off * m * q, hk - off, M.as<uint32_t>(), DM + 1, m,
                                   q, q, hprev - off, hk - off, p, R.as<uint32_t>()));
            }
            WR_TRY(pm_basis_rec(ctx, k > 0 ? R.as<uint32_t>() : F.as<uint32_t>(), d, m, q, p, d_deg, leaf, Mk, DMk));
            R.release();
            if (k == 0) {
                M = std::move(Mk);
                DM = DMk;
            } else {
                WR_CUDA(cudaMemcpyAsync(hd.data(), d_deg, sizeof(int32_t) * q, cudaMemcpyDeviceToHost, s));
                WR_CUDA(cudaStreamSynchronize(s));
                // starting degrees (0^n, 1^m): the smallest is 0
                const int64_t bound = (int64_t)*std::max_element(hd.begin(), hd.end());
                const int64_t DMn = std::max<int64_t>(0, std::min<int64_t>(DM + DMk, bound));
                DevBuf Mn;
                WR_TRY(dev_alloc(ctx, Mn, sizeof(uint32_t) * (size_t)(DMn + 2) * q * q));
                WR_CUDA(cudaMemsetAsync(Mn.ptr, 0, Mn.bytes, s));
                WR_TRY(polymat_mul(ctx, M.as<uint32_t>(), DM + 1, Mk.as<uint32_t>(), DMk + 1, q, q, q, 0, DMn + 1, p,
                                   Mn.as<uint32_t>()));
                M = std::move(Mn);
                DM = DMn;
            }
            hprev = hk;
        }
    } else {
        if (ctx->feed) WR_TRY(feed_wait(ctx, ctx->feed, L));  // PM-Basis reads the whole sequence
        WR_TRY(build_F(0, L));
        WR_TRY(pm_basis_rec(ctx, F.as<uint32_t>(), L, m, q, p, d_deg, leaf, M, DM));
    }
    if (DM > Dcap) return fail(WR_EINVAL, "sigma-basis degree cap too small");
    WR_CUDA(cudaMemsetAsync(d_P, 0, sizeof(uint32_t) * (Dcap + 1) * n * q, s));
    const unsigned g2 = (unsigned)std::min<int64_t>(((DM + 1) * n * q + 255) / 256, (int64_t)ctx->num_sms * 16);
    k_top_rows<<<g2, 256, 0, s>>>(M.as<uint32_t>(), DM, n, q, d_P);
    WR_LAUNCHED(ctx);
    WR_CUDA(cudaStreamSynchronize(s));
    return WR_OK;
}

wr_status det_valuation(wr_ctx *ctx, const uint32_t *d_G, int64_t n, int64_t T, uint32_t p, int64_t *val) {
    if (n <= 0) { *val = 0; return WR_OK; }
    if (n > 64 || T < 1 || T > 4096) return fail(WR_EINVAL, "det valuation: n in 1..64 and T in 1..4096");
    const ModP mp = make_modp(p);
    DevBuf g, out;
    WR_TRY(dev_alloc(ctx, g, sizeof(uint32_t) * n * n * T));
    WR_TRY(dev_alloc(ctx, out, sizeof(int64_t)));
    size_t smem = sizeof(uint32_t) * (T + (size_t)n * T) + sizeof(int) * 2 * n;
    if (smem > 200 * 1024) return fail(WR_EINVAL, "det valuation: precision too large");
    WR_CUDA(cudaFuncSetAttribute(k_valuation, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 48 * 1024)));
    k_valuation<<<1, VAL_THREADS, smem, ctx->stream>>>(d_G, g.as<uint32_t>(), (int)n, (int)T,
                                                       out.as<int64_t>(), mp);
    WR_LAUNCHED(ctx);
    WR_CUDA(cudaMemcpyAsync(val, out.ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    WR_CUDA(cudaStreamSynchronize(ctx->stream));
    return WR_OK;
}

wr_status rank_readout(wr_ctx *ctx, const uint32_t *d_P, const int32_t *d_deg, int m, int n, uint32_t p,
                       int64_t Dcap, Readout &out, std::vector<uint32_t> *gen) {
    const int q = m + n;
    cudaStream_t s = ctx->stream;
    DevBuf sel, delta;
    WR_TRY(dev_alloc(ctx, sel, sizeof(int32_t) * n));
    WR_TRY(dev_alloc(ctx, delta, sizeof(int32_t) * n));
    k_select<<<1, 64, 0, s>>>(d_deg, q, n, sel.as<int32_t>(), delta.as<int32_t>());
    WR_LAUNCHED(ctx);
    out.delta.assign(n, 0);
    WR_CUDA(cudaMemcpyAsync(out.delta.data(), delta.ptr, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    int64_t sd = 0, dmax = 0;
    for (int j = 0; j < n; j++) {
        sd += out.delta[j];
        dmax = std::max<int64_t>(dmax, out.delta[j]);
    }
    out.sum_delta = sd;
    out.dmax = dmax;
    // valuations of det P and det F (F_j(x) = x^delta_j P_j(1/x)); double the
    // precision until every pivot is found; coefficients past the degree are
    // zero, so T > n (dmax + 1) decides det = 0.
    int64_t vals[2] = {0, 0};
    for (int which = 0; which < 2; which++) {
        int64_t T = 8;
        for (;;) {
            DevBuf G;
            WR_TRY(dev_alloc(ctx, G, sizeof(uint32_t) * T * n * n));
            k_extract<<<blocks_for(T * n * n, 256), 256, 0, s>>>(d_P, n, q, sel.as<int32_t>(), delta.as<int32_t>(),
                                                                 T, which, Dcap, G.as<uint32_t>());
            WR_LAUNCHED(ctx);
            int64_t v = -1;
            WR_TRY(det_valuation(ctx, G.as<uint32_t>(), n, T, p, &v));
            if (v >= 0) { vals[which] = v; break; }
            if (T > (int64_t)n * (dmax + 1) + 2 || T >= 4096)
                return fail(WR_EPROBFAIL, "generator determinant vanishes (singular generator)");
            T *= 2;
        }
    }
    out.vP = vals[0];
    out.codeg = vals[1];
    out.deg_det = sd - vals[0];
    out.rank = out.deg_det - out.codeg;
    if (gen) {
        const int64_t T = dmax + 1;
        DevBuf G;
        WR_TRY(dev_alloc(ctx, G, sizeof(uint32_t) * T * n * n));
        k_extract<<<blocks_for(T * n * n, 256), 256, 0, s>>>(d_P, n, q, sel.as<int32_t>(), delta.as<int32_t>(),
                                                             T, 1, Dcap, G.as<uint32_t>());
        WR_LAUNCHED(ctx);
        gen->resize((size_t)T * n * n);
        WR_CUDA(cudaMemcpyAsync(gen->data(), G.ptr, sizeof(uint32_t) * gen->size(), cudaMemcpyDeviceToHost, s));
        WR_CUDA(cudaStreamSynchronize(s));
    }
    return WR_OK;
}

}  // namespace wr
