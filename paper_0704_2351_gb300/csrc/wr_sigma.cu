// sigma-basis of the block Wiedemann sequence and the rank readout
// (Section 2.3 "sigma-basis computations", Section 2.4 steps 3 and 4).
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

__global__ void k_init_basis(uint32_t *__restrict__ P, int n, int q, int32_t *__restrict__ deg,
                             uint32_t *__restrict__ qtop, int m, int *__restrict__ dmax) {
    for (int t = threadIdx.x; t < m * q || t < q; t += blockDim.x) {
        if (t < n) P[(size_t)t * q + t] = 1;  // P = [I_n | 0] at x^0
        if (t < q) deg[t] = t < n ? 0 : 1;
        if (t < m * q) {
            int a = t / q, c = t % q;
            qtop[t] = (c == n + a) ? 1u : 0u;  // Q = [0 | I_m] at x^0
        }
    }
    if (threadIdx.x == 0) *dmax = 1;
}

// E_acc[(i*m + a)*q + c] += sum_{t in tile} sum_r S[k0+i-t][a][r] P[t][r][c]
template <int KLAZY>
__global__ void k_window(const uint32_t *__restrict__ S, int64_t L, int m, int n, int q,
                         const uint32_t *__restrict__ P, int64_t k0, int bb, int TT, int CT,
                         const int *__restrict__ dmax_dev, unsigned long long *__restrict__ E_acc,
                         ModP mp) {
    extern __shared__ uint32_t sm[];
    const int64_t t0 = (int64_t)blockIdx.x * TT;
    const int c0 = blockIdx.y * CT;
    const int ct = min(CT, q - c0);
    const int dmax = *dmax_dev;
    if (t0 > dmax || t0 > k0 + bb - 1) return;
    const int tt_n = (int)min64(TT, min64(dmax + 1, k0 + bb) - t0);
    uint32_t *Ps = sm;                          // [TT][n][CT]
    uint32_t *Ss = sm + (size_t)TT * n * CT;    // [bb + TT - 1][m][n]
    const int mn = m * n;
    for (int i = threadIdx.x; i < tt_n * n * ct; i += blockDim.x) {
        int tl = i / (n * ct), rem = i % (n * ct), r = rem / ct, cl = rem % ct;
        Ps[(tl * n + r) * CT + cl] = P[((size_t)(t0 + tl) * n + r) * q + c0 + cl];
    }
    const int64_t smin = k0 - t0 - tt_n + 1;
    const int scount = bb + tt_n - 1;
    for (int i = threadIdx.x; i < scount * mn; i += blockDim.x) {
        int64_t s = smin + i / mn;
        Ss[i] = (s >= 0 && s < L) ? S[(size_t)s * mn + i % mn] : 0u;
    }
    __syncthreads();
    const int nout = bb * m * ct;
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int i = o / (m * ct), a = (o / ct) % m, cl = o % ct;
        unsigned long long acc = 0;
        int cnt = 0;
        for (int tl = 0; tl < tt_n; tl++) {
            const int64_t s = k0 + i - (t0 + tl);
            if (s < 0) break;
            const uint32_t *srow = Ss + (size_t)(s - smin) * mn + a * n;
            const uint32_t *pcol = Ps + (size_t)tl * n * CT + cl;
            for (int r = 0; r < n; r++) {
                acc += (unsigned long long)srow[r] * pcol[r * CT];
                if (++cnt == KLAZY) { acc = red64(acc, mp); cnt = 0; }
            }
        }
        acc = red64(acc, mp);
        if (acc) atomicAdd(&E_acc[((size_t)i * m + a) * q + c0 + cl], acc);
    }
}

// Local M-Basis over the window: one block.
// Shared layout: Es [bb][m][q], Ml [bb+1][q][q], D [m][q], Tff [q][q],
// Tp [m][q], and small vectors.
constexpr int LOCAL_THREADS = 512;

__global__ void __launch_bounds__(LOCAL_THREADS)
    k_local(int m, int n, int q, int bb, unsigned long long *__restrict__ E_acc,
            uint32_t *__restrict__ qtop, int32_t *__restrict__ deg_g, uint32_t *__restrict__ Ml_g,
            int32_t *__restrict__ degl_g, int *__restrict__ dmax_g, ModP mp) {
    extern __shared__ uint32_t sm[];
    uint32_t *Es = sm;                                   // bb*m*q
    uint32_t *Ml = Es + (size_t)bb * m * q;              // (bb+1)*q*q
    uint32_t *D = Ml + (size_t)(bb + 1) * q * q;         // m*q
    uint32_t *Tff = D + m * q;                           // q*q  (row j: transform of column j)
    uint32_t *Tp = Tff + q * q;                          // m*q  (Tp[t][j] = T[pc[t]][j])
    uint32_t *scl = Tp + m * q;                          // q
    uint32_t *sinv = scl + q;                            // q
    int *deg = (int *)(sinv + q);                        // q
    int *degl = deg + q;                                 // q
    int *ord = degl + q;                                 // q
    int *pc = ord + q;                                   // m
    int *pr = pc + m;                                    // m
    int *isp = pr + m;                                   // q (pivot flag)
    int *npiv = isp + q;                                 // 1
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;

    for (int i = tid; i < bb * m * q; i += nth) {
        unsigned long long v = E_acc[i];
        E_acc[i] = 0;
        uint32_t e = red64(v, mp);
        if (i < m * q) e = subm(e, qtop[i], mp);
        Es[i] = e;
    }
    for (int i = tid; i < (bb + 1) * q * q; i += nth) {
        int s = i / (q * q), rem = i % (q * q);
        Ml[i] = (s == 0 && rem / q == rem % q) ? 1u : 0u;
    }
    for (int c = tid; c < q; c += nth) {
        deg[c] = deg_g[c];
        degl[c] = 0;
    }
    __syncthreads();

    for (int i = 0; i < bb; i++) {
        // ---- elimination on Delta = Es[i] (warp 0)
        if (warp == 0) {
            for (int x = lane; x < m * q; x += 32) D[x] = Es[(size_t)i * m * q + x];
            for (int c = lane; c < q; c += 32) {
                int rk = 0;
                for (int c2 = 0; c2 < q; c2++)
                    rk += (deg[c2] < deg[c] || (deg[c2] == deg[c] && c2 < c)) ? 1 : 0;
                ord[rk] = c;
                scl[c] = 1;
                isp[c] = 0;
                for (int x = 0; x < q; x++) Tff[c * q + x] = (x == c) ? 1u : 0u;
            }
            __syncwarp();
            int np = 0;
            for (int oi = 0; oi < q; oi++) {
                const int j = ord[oi];
                for (int t = 0; t < np; t++) {
                    const int c = pc[t], r = pr[t];
                    const uint32_t dj = D[r * q + j];
                    if (dj == 0) continue;
                    const uint32_t dc = D[r * q + c];
                    __syncwarp();
                    for (int a = lane; a < m; a += 32)
                        D[a * q + j] = subm(mulm(dc, D[a * q + j], mp), mulm(dj, D[a * q + c], mp), mp);
                    for (int x = lane; x < q; x += 32)
                        Tff[j * q + x] = subm(mulm(dc, Tff[j * q + x], mp), mulm(dj, Tff[c * q + x], mp), mp);
                    if (lane == 0) scl[j] = mulm(scl[j], dc, mp);
                    __syncwarp();
                }
                bool nzr = false;
                for (int a = lane; a < m; a += 32) nzr |= D[a * q + j] != 0;
                // first nonzero row (m <= 32: one row per lane)
                unsigned bal = __ballot_sync(0xffffffffu, lane < m && D[lane * q + j] != 0);
                (void)nzr;
                if (bal) {
                    if (lane == 0) {
                        pc[np] = j;
                        pr[np] = __ffs(bal) - 1;
                        isp[j] = 1;
                    }
                    np++;
                }
                __syncwarp();
            }
            if (lane == 0) *npiv = np;
            for (int c = lane; c < q; c += 32) sinv[c] = invm(scl[c], mp);
            __syncwarp();
            // normalised transform restricted to pivot rows: Tp[t][j] = T[pc[t]][j]
            for (int x = lane; x < np * q; x += 32) {
                int t = x / q, j = x % q;
                uint32_t v = (j == pc[t]) ? 0u : mulm(Tff[j * q + pc[t]], sinv[j], mp);
                Tp[t * q + j] = v;
            }
            __syncwarp();
            // local degree bounds: column j now also holds multiples of the
            // pivot columns added to it, which may have a larger local degree
            int dnew[2];
            for (int k = 0; k < 2; k++) {
                const int j = lane + 32 * k;
                dnew[k] = 0;
                if (j < q) {
                    int d = degl[j];
                    for (int t = 0; t < np; t++)
                        if (Tp[t * q + j]) d = max(d, degl[pc[t]]);
                    dnew[k] = d;
                }
            }
            __syncwarp();
            for (int k = 0; k < 2; k++)
                if (lane + 32 * k < q) degl[lane + 32 * k] = dnew[k];
        }
        __syncthreads();
        const int np = *npiv;
        // ---- apply the transform to the rest of the window and to Ml (row-wise)
        //      new[j] = old[j] + sum_t Tp[t][j] old[pc[t]]
        {
            const int erows = (bb - i) * m;        // rows (i', a), i' in [i, bb)
            int dl = 0;
            for (int c = 0; c < q; c++) dl = max(dl, degl[c]);
            const int mrows = (dl + 1) * q;        // rows (s, x) of Ml, s <= max degl
            const int nrows = erows + mrows;
            for (int row = warp; row < nrows; row += nth / 32) {
                uint32_t *base = row < erows ? Es + ((size_t)i * m + row) * q
                                             : Ml + (size_t)(row - erows) * q;
                uint32_t v0 = lane < q ? base[lane] : 0u;
                uint32_t v1 = lane + 32 < q ? base[lane + 32] : 0u;
                uint32_t n0 = v0, n1 = v1;
                for (int t = 0; t < np; t++) {
                    const int c = pc[t];
                    const uint32_t oc = c < 32 ? __shfl_sync(0xffffffffu, v0, c)
                                               : __shfl_sync(0xffffffffu, v1, c - 32);
                    if (oc == 0) continue;
                    if (lane < q) n0 = addm(n0, mulm(Tp[t * q + lane], oc, mp), mp);
                    if (lane + 32 < q) n1 = addm(n1, mulm(Tp[t * q + lane + 32], oc, mp), mp);
                }
                if (lane < q) base[lane] = n0;
                if (lane + 32 < q) base[lane + 32] = n1;
            }
        }
        __syncthreads();
        // ---- multiply pivot columns by x: shift in the window and in Ml
        for (int w = tid; w < np * (m + q); w += nth) {
            const int t = w / (m + q), k = w % (m + q);
            const int c = pc[t];
            if (k < m) {
                const int a = k;
                for (int ii = bb - 1; ii > i; ii--)
                    Es[((size_t)ii * m + a) * q + c] = Es[((size_t)(ii - 1) * m + a) * q + c];
            } else {
                const int x = k - m;
                for (int s = degl[c] + 1; s > 0; s--)
                    Ml[((size_t)s * q + x) * q + c] = Ml[((size_t)(s - 1) * q + x) * q + c];
                Ml[(size_t)x * q + c] = 0;
            }
        }
        __syncthreads();
        for (int t = tid; t < np; t += nth) {
            deg[pc[t]] += 1;
            degl[pc[t]] += 1;
        }
        __syncthreads();
    }
    // ---- Qtop <- Qtop * Ml[bb]; write back
    for (int x = tid; x < m * q; x += nth) {
        const int a = x / q, c = x % q;
        unsigned long long acc = 0;
        for (int y = 0; y < q; y++) {
            acc += (unsigned long long)qtop[a * q + y] * Ml[((size_t)bb * q + y) * q + c];
            acc = red64(acc, mp);
        }
        D[x] = (uint32_t)acc;
    }
    __syncthreads();
    for (int x = tid; x < m * q; x += nth) qtop[x] = D[x];
    for (int x = tid; x < (bb + 1) * q * q; x += nth) Ml_g[x] = Ml[x];
    for (int c = tid; c < q; c += nth) {
        deg_g[c] = deg[c];
        degl_g[c] = degl[c];
    }
    if (tid == 0) {
        int d = 0;
        for (int c = 0; c < q; c++) d = max(d, deg[c]);
        *dmax_g = d;
    }
}

// P_new[t][r][c] = sum_{s <= min(t, degl[c])} sum_x P[t-s][r][x] Ml[s][x][c]
template <int KLAZY>
__global__ void k_apply(const uint32_t *__restrict__ P, uint32_t *__restrict__ Pn, int n, int q,
                        const uint32_t *__restrict__ Ml_g, const int32_t *__restrict__ degl_g, int bb,
                        int64_t Dbound, int TA, ModP mp) {
    extern __shared__ uint32_t sm[];
    uint32_t *Mls = sm;                               // (bb+1)*q*q
    uint32_t *Pss = Mls + (size_t)(bb + 1) * q * q;   // (TA + bb) * n * q
    __shared__ int degl[64];
    const int64_t t0 = (int64_t)blockIdx.x * TA;
    if (t0 > Dbound) return;
    const int ta = (int)min64(TA, Dbound + 1 - t0);
    for (int i = threadIdx.x; i < (bb + 1) * q * q; i += blockDim.x) Mls[i] = Ml_g[i];
    for (int i = threadIdx.x; i < q; i += blockDim.x) degl[i] = degl_g[i];
    const int64_t pbase = t0 - bb;  // Pss[u] holds P[pbase + u]
    const int nq = n * q;
    for (int i = threadIdx.x; i < (ta + bb) * nq; i += blockDim.x) {
        int64_t t = pbase + i / nq;
        Pss[i] = t >= 0 ? P[(size_t)t * nq + i % nq] : 0u;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < ta * nq; o += blockDim.x) {
        const int tl = o / nq, r = (o / q) % n, c = o % q;
        const int64_t t = t0 + tl;
        unsigned long long acc = 0;
        int cnt = 0;
        const int smax = (int)min64(degl[c], t);
        for (int s = 0; s <= smax; s++) {
            const uint32_t *prow = Pss + (size_t)(t - s - pbase) * nq + r * q;
            const uint32_t *mcol = Mls + (size_t)s * q * q + c;
            for (int x = 0; x < q; x++) {
                acc += (unsigned long long)prow[x] * mcol[x * q];
                if (++cnt == KLAZY) { acc = red64(acc, mp); cnt = 0; }
            }
        }
        Pn[(size_t)t * nq + r * q + c] = red64(acc, mp);
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

wr_status sigma_basis(wr_ctx *ctx, const uint32_t *d_S, int64_t L, int m, int n, uint32_t p,
                      uint32_t *d_P, int32_t *d_deg, int64_t Dcap) {
    if (m < 1 || n < 1 || m > 32 || n > 32) return fail(WR_EINVAL, "block sizes must be in 1..32");
    const int q = m + n;
    const ModP mp = make_modp(p);
    cudaStream_t s = ctx->stream;
    const size_t nq = (size_t)n * q;
    WR_CUDA(cudaMemsetAsync(d_P, 0, sizeof(uint32_t) * (Dcap + 1) * nq, s));
    DevBuf P2, qtop, Ml, degl, dmax, Eacc;
    WR_TRY(dev_alloc(ctx, P2, sizeof(uint32_t) * (Dcap + 1) * nq));
    WR_CUDA(cudaMemsetAsync(P2.ptr, 0, P2.bytes, s));
    WR_TRY(dev_alloc(ctx, qtop, sizeof(uint32_t) * m * q));
    WR_TRY(dev_alloc(ctx, degl, sizeof(int32_t) * q));
    WR_TRY(dev_alloc(ctx, dmax, sizeof(int)));
    k_init_basis<<<1, 256, 0, s>>>(d_P, n, q, d_deg, qtop.as<uint32_t>(), m, dmax.as<int>());
    WR_LAUNCHED(ctx);

    // chunk size: the local kernel's shared memory must fit
    const size_t budget = std::min<size_t>(ctx->smem_optin, 227 * 1024) - 1024;
    auto local_bytes = [&](int b) {
        return sizeof(uint32_t) * ((size_t)b * m * q + (size_t)(b + 1) * q * q + m * q + q * q + m * q + 2 * q) +
               sizeof(int) * (3 * q + 2 * m + q + 1);
    };
    int bmax = 64;
    while (bmax > 1 && local_bytes(bmax) > budget) bmax /= 2;
    // window tiles
    const int CT = std::min(q, 16);
    auto window_bytes = [&](int TT, int b) {
        return sizeof(uint32_t) * ((size_t)TT * n * CT + (size_t)(b + TT - 1) * m * n);
    };
    int TT = 64;
    while (TT > 1 && window_bytes(TT, bmax) > budget) TT /= 2;
    int TA = 16;
    auto apply_bytes = [&](int ta, int b) {
        return sizeof(uint32_t) * ((size_t)(b + 1) * q * q + (size_t)(ta + b) * nq);
    };
    while (TA > 1 && apply_bytes(TA, bmax) > budget) TA /= 2;
    if (apply_bytes(TA, bmax) > budget) return fail(WR_EINVAL, "block sizes too large for shared memory");

    WR_TRY(dev_alloc(ctx, Ml, sizeof(uint32_t) * (bmax + 1) * q * q));
    WR_TRY(dev_alloc(ctx, Eacc, sizeof(unsigned long long) * (size_t)bmax * m * q));
    WR_CUDA(cudaMemsetAsync(Eacc.ptr, 0, Eacc.bytes, s));
    const bool lazy16 = mp.lazy >= 16;
    auto *kwin = lazy16 ? k_window<16> : k_window<4>;
    auto *kapp = lazy16 ? k_apply<16> : k_apply<4>;
    WR_CUDA(cudaFuncSetAttribute(kwin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));
    WR_CUDA(cudaFuncSetAttribute(k_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));
    WR_CUDA(cudaFuncSetAttribute(kapp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));

    uint32_t *Pcur = d_P, *Pnext = P2.as<uint32_t>();
    int64_t Dbound = 1;
    for (int64_t k0 = 0; k0 < L; k0 += bmax) {
        const int bb = (int)std::min<int64_t>(bmax, L - k0);
        // window
        {
            dim3 grid((unsigned)((std::min(Dbound, k0 + bb - 1) + TT) / TT), (unsigned)((q + CT - 1) / CT));
            kwin<<<grid, 256, window_bytes(TT, bb), s>>>(d_S, L, m, n, q, Pcur, k0, bb, TT, CT,
                                                          dmax.as<int>(), Eacc.as<unsigned long long>(), mp);
            WR_LAUNCHED(ctx);
        }
        k_local<<<1, LOCAL_THREADS, local_bytes(bb), s>>>(m, n, q, bb, Eacc.as<unsigned long long>(),
                                                         qtop.as<uint32_t>(), d_deg, Ml.as<uint32_t>(),
                                                         degl.as<int32_t>(), dmax.as<int>(), mp);
        WR_LAUNCHED(ctx);
        const int64_t Dnew = std::min<int64_t>(Dbound + bb, Dcap);
        if (Dbound + bb > Dcap + 1) return fail(WR_EINVAL, "sigma-basis degree cap too small");
        kapp<<<(unsigned)((Dnew + TA) / TA), 256, apply_bytes(TA, bb), s>>>(
            Pcur, Pnext, n, q, Ml.as<uint32_t>(), degl.as<int32_t>(), bb, Dnew, TA, mp);
        WR_LAUNCHED(ctx);
        std::swap(Pcur, Pnext);
        Dbound = Dnew;
    }
    if (Pcur != d_P)
        WR_CUDA(cudaMemcpyAsync(d_P, Pcur, sizeof(uint32_t) * (Dbound + 1) * nq, cudaMemcpyDeviceToDevice, s));
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
