"""Pins of the CPU oracle to things other than itself (runs without a GPU).

Each test pins one oracle function to a fact the paper or the mathematics fixes:
published test vectors, brute force on tiny inputs, closed forms, invariants,
special cases that reduce to textbook routines.  Each is chosen so that a
plausible slip (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_0704_2351_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PRIMES = [65521, 1073741789, 2147483629]


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


# ---------------------------------------------------------------- random draws

def test_splitmix64_published_vector():
    """Pins the counter-based generator to SplitMix64's published outputs."""
    vals = [int(x[0]) for x in _rows("splitmix64.txt")]
    seed, expect = vals[0], vals[1:]
    golden = 0x9E3779B97F4A7C15
    got = [oracle.splitmix64((seed + k * golden) % 2**64) for k in range(len(expect))]
    assert got == expect


def test_derived_blocks_in_range_and_diagonals_nonzero():
    for p in PRIMES + [5]:
        X = oracle.derive_block(7, oracle.TAG_X, 50, 3, p)
        assert X.max() < p
        d = oracle.derive_diag(7, oracle.TAG_D1, 500, p)
        assert d.min() >= 1 and d.max() <= p - 1
    # tags give different streams
    assert not np.array_equal(oracle.derive_block(1, 1, 10, 2, 65521),
                              oracle.derive_block(1, 2, 10, 2, 65521))


# ---------------------------------------------------------------- primality

def _trial_div(n):
    if n < 2:
        return False
    f = 2
    while f * f <= n:
        if n % f == 0:
            return False
        f += 1
    return True


def test_miller_rabin_against_trial_division():
    for n in range(0, 20000):
        assert oracle.is_prime(n) == _trial_div(n), n
    # strong pseudoprimes to several bases and Carmichael numbers
    for n in [2047, 3277, 4033, 4681, 8321, 561, 1105, 1729, 2465, 25326001, 3215031751]:
        assert not oracle.is_prime(n), n
    for n in PRIMES + [65537, 2147483647, 4294967291]:
        assert oracle.is_prime(n) == _trial_div(n)


def test_primes_below_2_30():
    ps = oracle.primes_below(2**30, 4)
    assert len(ps) == 4 and all(_trial_div(p) for p in ps)
    for lo, hi in zip(ps[1:], ps[:-1]):
        assert all(not _trial_div(x) for x in range(lo + 1, hi))


# ---------------------------------------------------------------- elimination

def _brute_kernel_size(a, p):
    rows, cols = a.shape
    cnt = 0
    for v in itertools.product(range(p), repeat=cols):
        if not np.any(a.dot(np.array(v, dtype=np.int64)) % p):
            cnt += 1
    return cnt


@pytest.mark.parametrize("p", [5, 7])
def test_dense_rank_brute_force(p):
    """rank = cols - log_p |ker|, kernel counted by enumerating all vectors."""
    rng = np.random.default_rng(p)
    for _ in range(40):
        r, c = int(rng.integers(1, 5)), int(rng.integers(1, 5))
        a = rng.integers(-3, 4, size=(r, c))
        if rng.random() < 0.3 and r > 1:
            a[-1] = (2 * a[0] - a[1 % r])  # force a dependency sometimes
        k = _brute_kernel_size(a, p)
        assert p ** (c - oracle.rank_dense(a, p)) == k


def test_dense_rank_transpose_and_products():
    rng = np.random.default_rng(1)
    for p in PRIMES:
        for _ in range(10):
            r, c, k = int(rng.integers(2, 30)), int(rng.integers(2, 30)), int(rng.integers(0, 12))
            # product of a full-column-rank r x k and full-row-rank k x c has rank k
            k = min(k, r, c)
            U = np.triu(rng.integers(-3, 4, size=(r, k)), 0)
            for i in range(k):
                U[i, i] = 1
            V = np.tril(rng.integers(-3, 4, size=(k, c)), 0)
            for i in range(k):
                V[i, i] = -1
            P1, P2 = rng.permutation(r), rng.permutation(c)
            a = (U @ V)[P1][:, P2]
            assert oracle.rank_dense(a, p) == k
            assert oracle.rank_dense(a.T, p) == k


def test_det_dense_closed_forms():
    p = 1073741789
    rng = np.random.default_rng(2)
    # Vandermonde: det = prod_{i<j} (x_j - x_i)
    xs = rng.integers(0, p, size=6)
    V = np.array([[pow(int(x), j, p) for j in range(6)] for x in xs], dtype=object)
    expect = 1
    for i in range(6):
        for j in range(i + 1, 6):
            expect = expect * (int(xs[j]) - int(xs[i])) % p
    assert oracle.det_dense(V.astype(np.int64), p) == expect
    # product rule
    A = rng.integers(0, 1000, size=(5, 5))
    B = rng.integers(0, 1000, size=(5, 5))
    AB = (A.astype(object).dot(B.astype(object)) % p).astype(np.int64)
    assert oracle.det_dense(AB, p) == oracle.det_dense(A, p) * oracle.det_dense(B, p) % p


def test_sparse_rank_equals_dense():
    for t in range(30):
        rng = np.random.default_rng(100 + t)
        R, C = int(rng.integers(1, 60)), int(rng.integers(1, 60))
        A = synth.random_sparse(R, C, int(rng.integers(1, 5)), seed=t)
        for p in [5, 65521, 2147483629]:
            assert oracle.rank_sparse(A, p) == oracle.rank_dense(A.to_dense(), p)


def test_planted_rank_by_construction():
    for t in range(12):
        rng = np.random.default_rng(200 + t)
        R, C = int(rng.integers(2, 80)), int(rng.integers(2, 80))
        r = int(rng.integers(0, min(R, C) + 1))
        A = synth.planted_sparse(R, C, r, row_len=int(rng.integers(1, 7)), seed=t)
        for p in [3, 65521, 1073741789]:
            assert oracle.rank_dense(A.to_dense(), p) == r
            assert oracle.rank_sparse(A, p) == r


def test_config0_planted_rank_sparse_elimination():
    A = synth.config0()
    assert A.rank == 1500
    assert oracle.rank_sparse(A, synth.PRIME_C0) == 1500


# ---------------------------------------------------------------- black box

def _dense_mod(a, p):
    return np.asarray(a, dtype=object) % p


@pytest.mark.parametrize("side", [0, 1])
def test_blackbox_equals_dense_formula(side):
    """A~ = D1 A^T D2 A D1 (side 0) or D1 A D2 A^T D1 (side 1), checked against
    dense products with exact integers."""
    p = 2147483629
    A = synth.random_sparse(23, 17, 4, seed=3)
    Ad = A.to_dense().astype(object)
    N = A.cols if side == 0 else A.rows
    Mo = A.rows if side == 0 else A.cols
    rng = np.random.default_rng(4)
    d1 = rng.integers(1, p, size=N)
    d2 = rng.integers(1, p, size=Mo)
    v = rng.integers(0, p, size=(N, 3))
    D1 = np.diag(d1.astype(object))
    D2 = np.diag(d2.astype(object))
    if side == 0:
        At = D1.dot(Ad.T).dot(D2).dot(Ad).dot(D1)
    else:
        At = D1.dot(Ad).dot(D2).dot(Ad.T).dot(D1)
    expect = (At.dot(v.astype(object)) % p).astype(np.int64)
    got = oracle.blackbox_apply(A, p, side, d1.astype(np.uint32), d2.astype(np.uint32),
                                v.astype(np.uint32))
    assert np.array_equal(got.astype(np.int64), expect)
    # A~ is symmetric: u^T A~ v == v^T A~ u
    assert np.array_equal(At % p, At.T % p)


def test_csr_products_equal_dense():
    p = 65521
    A = synth.random_sparse(31, 19, 5, seed=9)
    x = np.random.default_rng(0).integers(0, p, size=(19, 4))
    y = np.random.default_rng(1).integers(0, p, size=(31, 4))
    Ad = A.to_dense().astype(object)
    assert np.array_equal(oracle.csr_mul(A, x, p).astype(np.int64),
                          (Ad.dot(x.astype(object)) % p).astype(np.int64))
    assert np.array_equal(oracle.csr_tmul(A, y, p).astype(np.int64),
                          (Ad.T.dot(y.astype(object)) % p).astype(np.int64))


def test_sequence_equals_dense_powers():
    p = 1073741789
    A = synth.random_sparse(14, 11, 3, seed=5)
    st = oracle.Setup(A, p, 3, 2, seed=77)
    S = oracle.sequence(A, st, L=7)
    Ad = A.to_dense().astype(object)
    D1 = np.diag(st.D1.astype(object))
    D2 = np.diag(st.D2.astype(object))
    At = D1.dot(Ad.T).dot(D2).dot(Ad).dot(D1) % p
    v = st.Y.astype(object)
    for i in range(7):
        assert np.array_equal(S[i].astype(np.int64), (st.X.astype(object).T.dot(v) % p).astype(np.int64))
        v = At.dot(v) % p


def test_symmetric_projection_gives_symmetric_terms():
    """With X = Y the terms Y^T A~^i Y are symmetric because A~ is (Section 2.3)."""
    p = 65521
    A = synth.random_sparse(40, 30, 4, seed=6)
    st = oracle.Setup(A, p, 4, 4, seed=3, symmetric=True)
    S = oracle.sequence(A, st, L=10)
    for i in range(10):
        assert np.array_equal(S[i], S[i].T)


# ---------------------------------------------------------------- Berlekamp-Massey

def test_bm_fibonacci():
    p = 65521
    s = [0, 1]
    for _ in range(30):
        s.append((s[-1] + s[-2]) % p)
    L, f = oracle.berlekamp_massey(np.array(s, dtype=np.uint32), p)
    assert L == 2
    assert [int(c) for c in f] == [p - 1, p - 1, 1]  # x^2 - x - 1


def test_bm_diagonal_minpoly_closed_form():
    """s_k = sum_i w_i lambda_i^k with distinct lambda, w != 0 has minimal
    polynomial prod (x - lambda_i)."""
    p = 1073741789
    rng = np.random.default_rng(8)
    for d in [1, 3, 7, 12]:
        lam = rng.choice(np.arange(1, 10**6), size=d, replace=False)
        w = rng.integers(1, p, size=d)
        s = [sum(int(w[i]) * pow(int(lam[i]), k, p) for i in range(d)) % p for k in range(2 * d + 4)]
        L, f = oracle.berlekamp_massey(np.array(s, dtype=np.uint32), p)
        expect = [1]
        for l in lam:
            expect = [(a - int(l) * b) % p for a, b in zip([0] + expect, expect + [0])]
        assert L == d and [int(c) for c in f] == expect


def test_bm_length_equals_hankel_rank():
    p = 65521
    rng = np.random.default_rng(9)
    for d in [2, 5, 9]:
        coef = rng.integers(0, p, size=d)
        s = list(rng.integers(0, p, size=d))
        for k in range(d, 4 * d):
            s.append(int(sum(int(coef[j]) * int(s[k - 1 - j]) for j in range(d)) % p))
        L, _ = oracle.berlekamp_massey(np.array(s, dtype=np.uint32), p)
        h = 2 * d
        H = np.array([[s[i + j] for j in range(h)] for i in range(h)], dtype=np.int64)
        assert L == oracle.rank_dense(H, p)


# ---------------------------------------------------------------- sigma-basis

def _random_seq(rng, L, m, n, p):
    return rng.integers(0, p, size=(L, m, n)).astype(np.uint32)


@pytest.mark.parametrize("m,n", [(1, 1), (2, 3), (3, 2), (4, 4)])
def test_mbasis_is_sigma_basis(m, n):
    """H M = 0 mod x^L with H = [S | -I], and det M = c x^{mL} (c != 0): every
    order adds exactly m to the degree of the determinant."""
    p = 65521
    rng = np.random.default_rng(m * 10 + n)
    L = 12
    S = _random_seq(rng, L, m, n, p)
    M, deg = oracle.mbasis(S, p)
    q = m + n
    H = np.zeros((L, m, q), dtype=np.int64)
    H[:, :, :n] = S
    H[0, :, n:] = (-np.eye(m, dtype=np.int64)) % p
    HM = oracle.polymat_mul(H, M.astype(np.int64), p, trunc=L)
    assert not HM.any()
    # determinant degree: sum of shifted degrees = sum of shifts + m L
    assert int(deg.sum()) == m + m * L
    # det M(x) = c x^{mL}: det M(a) / det M(b) = (a/b)^{mL}
    D = M.shape[0] - 1
    a, b = 12345, 777
    da = oracle.load().or_det_poly_eval(oracle._p(np.ascontiguousarray(M)), q, D, a, p)
    db = oracle.load().or_det_poly_eval(oracle._p(np.ascontiguousarray(M)), q, D, b, p)
    assert da != 0 and db != 0
    assert da * pow(db, p - 2, p) % p == pow(a * pow(b, p - 2, p) % p, m * L, p)


def test_mbasis_scalar_reduces_to_berlekamp_massey():
    p = 1073741789
    A = synth.random_sparse(30, 25, 3, seed=11)
    st = oracle.Setup(A, p, 1, 1, seed=5)
    S = oracle.sequence(A, st)
    M, deg = oracle.mbasis(S, p)
    cols, delta, P, F = oracle.select_generator(M, deg, 1)
    Lc, f = oracle.berlekamp_massey(S.ravel(), p)
    g = F[: delta[0] + 1, 0, 0].astype(object)
    g = [int(c) * pow(int(g[-1]), p - 2, p) % p for c in g]  # monic
    assert delta[0] == Lc and g == [int(c) for c in f]


@pytest.mark.parametrize("m,n", [(2, 2), (3, 2), (2, 4)])
def test_generator_annihilates_and_degree_is_hankel_rank(m, n):
    """Sum_k S_{i+k} F_k[:, j] = 0 for i + delta_j <= L - 1, and deg det F equals
    the rank of the block Hankel matrix [S_{i+j}] (the dimension of the Krylov
    space the sequence sees)."""
    p = 65521
    A = synth.random_sparse(25, 20, 3, seed=m * 7 + n)
    st = oracle.Setup(A, p, m, n, seed=9)
    S = oracle.sequence(A, st)
    L = S.shape[0]
    M, deg = oracle.mbasis(S, p)
    out = oracle.rank_readout(M, deg, n, p)
    F, delta = out["F"], out["delta"]
    for j in range(n):
        for i in range(L - int(delta[j])):
            acc = np.zeros(m, dtype=object)
            for k in range(int(delta[j]) + 1):
                acc = acc + S[i + k].astype(object).dot(F[k, :, j].astype(object))
            assert not np.any(acc % p)
    k1 = -(-st.N // m) + 1     # k1 m >= N rows, k2 n >= N columns, k1 + k2 - 1 = L
    k2 = L + 1 - k1
    Hk = np.block([[S[i + j].astype(np.int64) for j in range(k2)] for i in range(k1)])
    assert out["deg_det"] == oracle.rank_dense(Hk, p)


# ---------------------------------------------------------------- det valuation

def test_det_valuation_planted():
    """G = U diag(x^e) V with U(0), V(0) invertible has v_x(det G) = sum e."""
    p = 65521
    rng = np.random.default_rng(12)
    for t in range(20):
        n = int(rng.integers(1, 5))
        e = rng.integers(0, 4, size=n)
        U = rng.integers(0, p, size=(3, n, n))
        V = rng.integers(0, p, size=(3, n, n))
        U[0] = np.triu(U[0], 1) + np.eye(n, dtype=np.int64)  # invertible constant term
        V[0] = np.tril(V[0], -1) + np.eye(n, dtype=np.int64)
        Dg = np.zeros((int(e.max()) + 1, n, n), dtype=np.int64)
        for i in range(n):
            Dg[int(e[i]), i, i] = 1
        G = oracle.polymat_mul(oracle.polymat_mul(U, Dg, p), V, p)
        assert oracle.det_valuation(G.astype(np.uint32), p) == int(e.sum())


def test_det_valuation_matches_interpolated_determinant():
    p = 65521
    rng = np.random.default_rng(13)
    for t in range(15):
        n = int(rng.integers(1, 4))
        D = int(rng.integers(0, 4))
        G = rng.integers(0, p, size=(D + 1, n, n))
        G[0] = 0 if rng.random() < 0.5 else G[0]  # force x | G sometimes
        if rng.random() < 0.5 and D >= 1:
            G[1, 0] = 0
        det = oracle.det_poly(G.astype(np.uint32), p)
        nz = np.nonzero(det)[0]
        v = oracle.det_valuation(G.astype(np.uint32), p)
        if len(nz) == 0:
            assert v is None
        else:
            assert v == int(nz[0])


# ---------------------------------------------------------------- rank

def test_wiedemann_rank_equals_elimination_many_shapes():
    """The Monte Carlo rank (Section 2.5) equals the elimination rank."""
    bad = 0
    for t in range(25):
        rng = np.random.default_rng(300 + t)
        R, C = int(rng.integers(3, 90)), int(rng.integers(3, 90))
        r = int(rng.integers(0, min(R, C) + 1))
        A = synth.planted_sparse(R, C, r, row_len=int(rng.integers(1, 6)), seed=t)
        for (m, n) in [(1, 1), (2, 2), (3, 5), (8, 8)]:
            for p in PRIMES:
                out = oracle.rank_wiedemann(A, p, m, n, seed=4000 + t)
                if out["rank"] != r:
                    bad += 1
    assert bad == 0


def test_codeg_closed_form_generic():
    """For the generic preconditioned singular A~ (N x N, rank r):
    det F = x^{min(n, N - r)} g with g(0) != 0."""
    p = 1073741789
    for t in range(6):
        rng = np.random.default_rng(500 + t)
        R, C = int(rng.integers(20, 60)), int(rng.integers(20, 60))
        N = min(R, C)
        r = int(rng.integers(1, N))
        A = synth.planted_sparse(R, C, r, row_len=4, seed=t)
        for n in [1, 2, 4]:
            out = oracle.rank_wiedemann(A, p, n, n, seed=t)
            assert out["codeg"] == min(n, N - r)
            assert out["rank"] == r


def test_rank_of_transpose_and_both_sides():
    p = 65521
    A = synth.planted_sparse(70, 50, 33, row_len=4, seed=21)
    At = A.transpose()
    for side in [0, 1]:
        assert oracle.rank_wiedemann(A, p, 2, 2, seed=1, side=side)["rank"] == 33
        assert oracle.rank_wiedemann(At, p, 2, 2, seed=1, side=side)["rank"] == 33


def test_degenerate_cases():
    p = 65521
    Z = synth.csr_from_coo(5, 4, np.zeros(0), np.zeros(0), np.zeros(0))
    assert oracle.rank_wiedemann(Z, p, 1, 1, seed=1)["rank"] == 0
    assert oracle.rank_wiedemann(Z, p, 2, 2, seed=1)["rank"] == 0
    one = synth.dense_to_csr(np.array([[0, 1], [0, 0]]))
    assert oracle.rank_wiedemann(one, p, 1, 1, seed=1)["rank"] == 1
    full = synth.dense_to_csr(np.eye(6, dtype=np.int64))
    assert oracle.rank_wiedemann(full, p, 2, 2, seed=1)["rank"] == 6


def test_config0_wiedemann_scalar():
    A = synth.config0()
    out = oracle.rank_wiedemann(A, synth.PRIME_C0, 1, 1, seed=synth.SEED_BASE)
    assert out["rank"] == 1500
    assert out["S"].shape == (3602, 1, 1)


# ---------------------------------------------------------------- chain complexes

def test_chain_pair_invariants():
    """d o d = 0 over Z (exact integer product) and
    rank(d_n) + rank(d_{n+1}) <= dim C_n (Section 1.1, homology)."""
    for t in range(4):
        c_n = [40, 75, 120, 300][t]
        d_n, d_n1 = synth.chain_pair(c_n, seed=t, homology=t)
        assert d_n.cols == c_n and d_n1.rows == c_n
        prod = synth.spmul(d_n, d_n1)
        assert prod.nnz == 0
        p = 1073741789
        rn = oracle.rank_sparse(d_n, p)
        rn1 = oracle.rank_sparse(d_n1, p)
        assert rn == d_n.rank and rn1 == d_n1.rank
        assert rn + rn1 <= c_n
        assert c_n - rn - rn1 >= min(t, 1) if t else True


# ---------------------------------------------------------------- paper tables

def test_table_res_consistency():
    """Table tab:res: ker = n - rank (GL7d15's printed ker is garbled), and the
    chain invariants: GL7d(k+1)'s column count is GL7dk's row count, and
    rank(d_k) + rank(d_{k+1}) <= n_k."""
    rows = _rows("gl7_table_res.txt")
    tab = {r[0]: dict(omega=int(r[1]), n=int(r[2]), m=int(r[3]), rank=int(r[4]), ker=int(r[5]))
           for r in rows}
    for name, e in tab.items():
        if name == "GL7d15":
            assert e["n"] - e["rank"] == 328218 and e["ker"] == 28218
        else:
            assert e["ker"] == e["n"] - e["rank"], name
    names = [r[0] for r in rows]
    for a, b in zip(names, names[1:]):
        assert tab[b]["m"] == tab[a]["n"]
        assert tab[a]["rank"] + tab[b]["rank"] <= tab[a]["n"]
        assert tab[a]["n"] - tab[a]["rank"] - tab[b]["rank"] in (0, 1)


def test_table_rtime_iteration_rule():
    """Table tab:r-time: iter[p] = ceil(2 + 2 r / p) and iter[1] = 2 + 2 r.
    With r = N this is the sequence length the oracle uses for m = n = p."""
    for name, r, it1, itp, pp in _rows("gl7_table_rtime.txt"):
        r, it1, itp, pp = int(r), int(it1), int(itp), int(pp)
        assert it1 == 2 + 2 * r
        assert itp == -(-(2 * pp + 2 * r) // pp)
        if r % pp == 0:
            assert oracle.seq_length(r, pp, pp) == itp
    assert oracle.seq_length(1800, 1, 1) == 3602


@pytest.mark.parametrize("side", [0, 1])
def test_blackbox_apply_rows_equals_full_application(side):
    """The row-by-row spot check equals the whole application (itself pinned
    to dense products), on both sides, with heavy rows and columns."""
    p = 2147483629
    A = synth.planted_sparse(140, 120, 100, row_len=6, seed=13 + side)
    rng = np.random.default_rng(side)
    N = A.cols if side == 0 else A.rows
    M = A.rows if side == 0 else A.cols
    d1 = oracle.derive_diag(9, 3, N, p)
    d2 = oracle.derive_diag(9, 4, M, p)
    v = rng.integers(0, p, size=(N, 5)).astype(np.uint32)
    full = oracle.blackbox_apply(A, p, side, d1, d2, v)
    rows = rng.choice(N, 25, replace=False)
    assert np.array_equal(oracle.blackbox_apply_rows(A, p, side, d1, d2, v, rows), full[rows])


# ---------------------------------------------------------------------------
# early termination (reading of Section 4's remark; no GPU)
# ---------------------------------------------------------------------------

def _generator(S, p, n):
    M, deg = oracle.mbasis(S, p)
    return oracle.rank_readout(M, deg, n, p)


@pytest.mark.parametrize("m,R,C,r,seed", [(1, 70, 60, 25, 1), (2, 90, 80, 30, 2), (4, 160, 150, 50, 3),
                                          (3, 120, 110, 70, 4), (2, 100, 90, 89, 5)])
def test_early_termination_gives_the_full_generator(m, R, C, r, seed):
    """Stopping at the quiet point keeps the generator of all L terms bit for
    bit: the candidates' columns are final once they annihilate the quiet
    orders; a rank-deficient matrix reaches the point well before L (about
    2r/m + quiet orders), a nearly full-rank one may not reach it at all."""
    p = 1073741789
    A = synth.planted_sparse(R, C, r, row_len=5, seed=seed)
    st = oracle.Setup(A, p, m, m, seed=seed)
    S = oracle.sequence(A, st)
    L = S.shape[0]
    k = oracle.early_termination_point(S, p, chunk=8, quiet=8)
    if k is None:  # no room for the quiet orders before L (nearly full rank): all L terms
        assert r > min(R, C) - 8
        k = L
    assert k <= L
    full, short = _generator(S, p, m), _generator(S[:k], p, m)
    assert short["rank"] == full["rank"] == r
    assert np.array_equal(short["delta"], full["delta"]) and np.array_equal(short["F"], full["F"])
    if r < min(R, C) // 2:
        assert k < L - (min(R, C) - r) // (2 * m)


def test_early_termination_never_stops_on_a_sequence_without_a_short_generator():
    """A random sequence has no generator of degree below L/2 per column, so
    no chunk of the candidates is quiet."""
    p = 65521
    rng = np.random.default_rng(9)
    for m in [1, 2, 4]:
        S = rng.integers(0, p, size=(64, m, m)).astype(np.uint32)
        assert oracle.early_termination_point(S, p, chunk=8, quiet=8) is None


def test_early_termination_point_is_where_a_planted_mistake_shows():
    """A pin against a weaker criterion: counting a chunk as quiet without
    checking the candidates' residuals would stop at the first chunks of any
    sequence; the reading's check keeps the stop after the generator's degree."""
    p = 1073741789
    A = synth.planted_sparse(120, 110, 40, row_len=5, seed=12)
    st = oracle.Setup(A, p, 2, 2, seed=12)
    S = oracle.sequence(A, st)
    k = oracle.early_termination_point(S, p, chunk=4, quiet=4)
    full = _generator(S, p, 2)
    # the generator's degree max(delta) orders at least must have been seen
    assert k >= int(np.max(full["delta"]))


# ---------------------------------------------------------------------------
# two terms per application of A~ (the identities the device's symmetric and
# paired generic modes compute), from oracle primitives
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("side,m", [(0, 3), (1, 2), (0, 1)])
def test_two_terms_per_application_identities(side, m):
    """A~ = D1 A^T D2 A D1 is symmetric, so with U_k = A~^k X, V_k = A~^k Y:
    X^T A~^(2k) Y = U_k^T V_k and X^T A~^(2k+1) Y = (A D1 U_k)^T D2 (A D1 V_k)
    (rows side: A^T and A swap).  Checked against the literal sequence for
    independent X and Y (and X = Y), k = 0..6."""
    p = 1073741789
    A = synth.planted_sparse(70, 60, 45, row_len=4, seed=side * 10 + m)
    for symmetric in [False, True]:
        st = oracle.Setup(A, p, m, m, seed=5 + m, side=side, symmetric=symmetric)
        S = oracle.sequence(A, st, 14)
        U = st.X.astype(np.uint32)
        V = st.Y.astype(np.uint32)

        def half(W):  # A D1 W (columns side) or A^T D1 W (rows side)
            D1W = (st.D1.astype(object)[:, None] * W.astype(object)) % p
            return (oracle.csr_mul(A, D1W.astype(np.uint32), p) if side == 0
                    else oracle.csr_tmul(A, D1W.astype(np.uint32), p)).astype(object)

        for k in range(7):
            even = (U.astype(object).T.dot(V.astype(object))) % p
            assert np.array_equal(even.astype(np.uint64), S[2 * k].astype(np.uint64)), (k, "even")
            HU, HV = half(U), half(V)
            odd = (HU.T.dot(st.D2.astype(object)[:, None] * HV)) % p
            assert np.array_equal(odd.astype(np.uint64), S[2 * k + 1].astype(np.uint64)), (k, "odd")
            U = oracle.blackbox_apply(A, p, st.side, st.D1, st.D2, U)
            V = oracle.blackbox_apply(A, p, st.side, st.D1, st.D2, V)


def _poly_eval(P, x0, p):
    """P(x0) mod p for a polynomial matrix P ([deg+1, r, c]) by Horner's rule."""
    acc = np.zeros(P.shape[1:], dtype=object)
    for k in range(P.shape[0] - 1, -1, -1):
        acc = (acc * x0 + P[k].astype(object)) % p
    return acc


@pytest.mark.parametrize("p", [65521, 1073741789, 2147483629])
def test_polymat_mul_is_a_ring_homomorphism_image(p):
    """polymat_mul (the product PM-Basis needs): at random points x0 the
    product's value is the product of the values, C(x0) = A(x0) B(x0) mod p
    (a wrong shift, a dropped or transposed term breaks it at almost every
    point); the identity and x^k are neutral and shifting factors; and the
    scalar powers of (1 + x) give the binomial coefficients mod p."""
    rng = np.random.default_rng(p % 97)
    for (da, db, r, s, t) in [(1, 1, 1, 1, 1), (5, 3, 2, 3, 4), (17, 9, 3, 2, 3), (4, 12, 1, 5, 2)]:
        A = rng.integers(0, p, size=(da, r, s))
        B = rng.integers(0, p, size=(db, s, t))
        C = oracle.polymat_mul(A, B, p)
        assert C.shape == (da + db - 1, r, t)
        for x0 in rng.integers(0, p, size=4):
            lhs = _poly_eval(C, int(x0), p)
            rhs = _poly_eval(A, int(x0), p).dot(_poly_eval(B, int(x0), p)) % p
            assert np.array_equal(lhs, rhs)
        # truncation keeps the low coefficients
        assert np.array_equal(oracle.polymat_mul(A, B, p, trunc=3)[:3], C[:3])
    A = rng.integers(0, p, size=(6, 3, 3))
    I = np.eye(3, dtype=np.int64)[None]
    assert np.array_equal(oracle.polymat_mul(A, I, p), A % p)
    xk = np.zeros((4, 3, 3), np.int64)
    xk[3] = np.eye(3, dtype=np.int64)
    assert np.array_equal(oracle.polymat_mul(A, xk, p)[3:], A % p)
    assert not oracle.polymat_mul(A, xk, p)[:3].any()
    P = np.ones((1, 1, 1), np.int64)
    one_x = np.ones((2, 1, 1), np.int64)
    for _ in range(10):
        P = oracle.polymat_mul(P, one_x, p)
    assert [int(v) for v in P[:, 0, 0]] == [math.comb(10, k) % p for k in range(11)]


@pytest.mark.parametrize("p", [65521, 2147483629, 2147483647])
def test_project_is_the_exact_product_reduced(p):
    """project(X, V) = X^T V mod p (Section 2.3's dot products), against Python
    integers: with every residue p - 1 a 64-bit accumulator that is not reduced
    wraps after 4 rows at p near 2^31, so the row counts here would show it;
    a transposed operand changes the shape or the values."""
    rng = np.random.default_rng(p % 101)
    for N, m, n in [(1, 1, 1), (5, 3, 2), (4097, 4, 7), (70001, 2, 3)]:
        for kind in ["random", "top"]:
            X = rng.integers(0, p, size=(N, m)) if kind == "random" else np.full((N, m), p - 1)
            V = rng.integers(0, p, size=(N, n)) if kind == "random" else np.full((N, n), p - 1)
            S = oracle.project(X.astype(np.uint32), V.astype(np.uint32), p)
            ref = (X.astype(object).T.dot(V.astype(object))) % p
            assert S.shape == (m, n)
            assert np.array_equal(S.astype(np.int64), ref.astype(np.int64))
    # all p - 1: (p - 1)^2 N = N mod p
    N = 70001
    S = oracle.project(np.full((N, 2), p - 1, np.uint32), np.full((N, 2), p - 1, np.uint32), p)
    assert (S == N % p).all()


def test_side_choice_makes_N_the_smaller_dimension():
    """Section 2.3: A~ is formed on the smaller side, so N = min(rows, cols)
    under the automatic choice; an explicit side is kept."""
    assert oracle.choose_side(10, 7) == oracle.SIDE_COLS
    assert oracle.choose_side(7, 10) == oracle.SIDE_ROWS
    assert oracle.choose_side(8, 8) == oracle.SIDE_COLS
    assert oracle.choose_side(10, 7, oracle.SIDE_ROWS) == oracle.SIDE_ROWS
    for R, C in [(60, 45), (45, 60)]:
        A = synth.random_sparse(R, C, 4, seed=R)
        st = oracle.Setup(A, 65521, 2, 3, seed=1)
        assert st.N == min(R, C) and st.M == max(R, C)
        assert st.Y.shape == (st.N, 3)
