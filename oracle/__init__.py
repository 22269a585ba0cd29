"""CPU oracle for the block Wiedemann rank path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
leg import this package.  The CUDA library (paper_0704_2351_gb300) never
imports it, and nothing in it comes from the CUDA library: the two share only
the seeded input generators of paper_0704_2351_gb300.synth, which hold no
arithmetic of the method.

The heavy loops are plain C (oracle.c, built by build()); this module holds
the glue and the rank readout.  What each function computes, and where the
paper defines it:

* sequence()            S_i = X^T A~^i Y mod p, i < L           (Section 2.2; Section 2.5 step 2)
* blackbox_apply()      A~ = D1 A^T D2 A D1 (or D1 A D2 A^T D1)   (Section 2.3, Section 2.5 step 1)
* blackbox_apply_rows() selected rows of A~ v, one at a time      (same; spot checks at full size)
* mbasis()              sigma-basis of [S(x) | -I]               (Section 2.4 "sigma-basis computations")
* generator()           minimal right matrix generator F          (Section 2.5 step 3)
* rank_readout()        r = deg det F - codeg det F              (Section 2.5 step 4)
* early_termination_point()  first order count after which the generator
                        candidates have been quiet for `quiet` orders (Section 4's early
                        termination; the criterion is a reading, stated in the function)
* rank_dense/sparse()   rank_p by Gaussian elimination (definition of the rank)
* berlekamp_massey()    scalar minimal polynomial                (Section 1.2, Wiedemann)

Parity is pinned (tests/test_oracle_pins.py) by brute force on tiny inputs,
closed forms and invariants; see each test for what it pins.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

TAG_X, TAG_Y, TAG_D1, TAG_D2 = 1, 2, 3, 4
SIDE_COLS, SIDE_ROWS = 0, 1


def lib_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load():
    global _LIB
    if _LIB is not None:
        return _LIB
    build()
    lib = ctypes.CDLL(lib_path())
    u64, i64, i32, u32p, i64p, i32p = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    vp = ctypes.c_void_p
    lib.or_is_prime_u32.argtypes = [u64]; lib.or_is_prime_u32.restype = i32
    lib.or_splitmix64.argtypes = [u64]; lib.or_splitmix64.restype = u64
    lib.or_hash.argtypes = [u64, u64, u64]; lib.or_hash.restype = u64
    lib.or_derive_block.argtypes = [u64, u64, i64, i64, u64, vp]
    lib.or_derive_diag.argtypes = [u64, u64, i64, u64, vp]
    lib.or_csr_mul.argtypes = [i64, i64, vp, vp, vp, u64, i64, vp, vp]
    lib.or_csr_tmul.argtypes = [i64, i64, vp, vp, vp, u64, i64, vp, vp]
    lib.or_csr_transpose.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp]
    lib.or_blackbox_apply.argtypes = [i64, i64, vp, vp, vp, u64, i32, vp, vp, i64, vp]
    lib.or_project.argtypes = [i64, i64, i64, vp, vp, u64, vp]
    lib.or_sequence.argtypes = [i64, i64, vp, vp, vp, u64, i32, vp, vp, i64, i64, vp, vp, i64, vp, vp]
    lib.or_rank_dense.argtypes = [i64, i64, vp, u64]; lib.or_rank_dense.restype = i64
    lib.or_det_dense.argtypes = [i64, vp, u64]; lib.or_det_dense.restype = u64
    lib.or_rank_sparse.argtypes = [i64, i64, vp, vp, vp, u64]; lib.or_rank_sparse.restype = i64
    lib.or_berlekamp_massey.argtypes = [vp, i64, u64, vp]; lib.or_berlekamp_massey.restype = i64
    lib.or_mbasis.argtypes = [vp, i64, i64, i64, u64, i64, vp, vp]; lib.or_mbasis.restype = i32
    lib.or_det_valuation.argtypes = [vp, i64, i64, u64]; lib.or_det_valuation.restype = i64
    lib.or_det_poly_eval.argtypes = [vp, i64, i64, u64, u64]; lib.or_det_poly_eval.restype = u64
    lib.or_residue.argtypes = [i64, u64]; lib.or_residue.restype = u64
    lib.or_mulmod.argtypes = [u64, u64, u64]; lib.or_mulmod.restype = u64
    lib.or_invmod.argtypes = [u64, u64]; lib.or_invmod.restype = u64
    _LIB = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
# primes and random draws
# ---------------------------------------------------------------------------

def is_prime(n: int) -> bool:
    return bool(load().or_is_prime_u32(int(n)))


def primes_below(bound: int, count: int):
    out, x = [], bound - 1
    while len(out) < count and x > 2:
        if is_prime(x):
            out.append(x)
        x -= 1
    return out


def splitmix64(x: int) -> int:
    return int(load().or_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def derive_block(seed: int, tag: int, rows: int, width: int, p: int) -> np.ndarray:
    out = np.empty(rows * width, dtype=np.uint32)
    load().or_derive_block(seed, tag, rows, width, p, _p(out))
    return out.reshape(rows, width)


def derive_diag(seed: int, tag: int, length: int, p: int) -> np.ndarray:
    out = np.empty(length, dtype=np.uint32)
    load().or_derive_diag(seed, tag, length, p, _p(out))
    return out


# ---------------------------------------------------------------------------
# sparse products and the black box
# ---------------------------------------------------------------------------

def _csr_args(A):
    rp = _c(A.rowptr, np.int64)
    ci = _c(A.colidx, np.int32)
    va = _c(A.vals, np.int32)
    return rp, ci, va


def csr_mul(A, x: np.ndarray, p: int) -> np.ndarray:
    x = _c(x, np.uint32).reshape(A.cols, -1)
    w = x.shape[1]
    y = np.empty((A.rows, w), dtype=np.uint32)
    rp, ci, va = _csr_args(A)
    load().or_csr_mul(A.rows, A.cols, _p(rp), _p(ci), _p(va), p, w, _p(x), _p(y))
    return y


def csr_tmul(A, x: np.ndarray, p: int) -> np.ndarray:
    x = _c(x, np.uint32).reshape(A.rows, -1)
    w = x.shape[1]
    y = np.empty((A.cols, w), dtype=np.uint32)
    rp, ci, va = _csr_args(A)
    load().or_csr_tmul(A.rows, A.cols, _p(rp), _p(ci), _p(va), p, w, _p(x), _p(y))
    return y


def choose_side(rows: int, cols: int, side: Optional[int] = None) -> int:
    """AUTO: the smaller dimension is N (Section 2.3: A~ of the form A^T A)."""
    if side is not None:
        return side
    return SIDE_COLS if rows >= cols else SIDE_ROWS


def seq_length(N: int, m: int, n: int) -> int:
    """L = ceil(N/m) + ceil(N/n) + 2 (Section 2.5 step 2: 2n/s + O(1) terms)."""
    return -(-N // m) + -(-N // n) + 2


class Setup:
    """The random choices of one run: X, Y, D1, D2 derived from the seed."""

    def __init__(self, A, p: int, m: int, n: int, seed: int, side: Optional[int] = None,
                 symmetric: bool = False):
        self.side = choose_side(A.rows, A.cols, side)
        self.N = A.cols if self.side == SIDE_COLS else A.rows
        self.M = A.rows if self.side == SIDE_COLS else A.cols
        self.p, self.m, self.n, self.seed = p, m, n, seed
        self.Y = derive_block(seed, TAG_Y, self.N, n, p)
        if symmetric:
            assert m == n
            self.X = self.Y.copy()
        else:
            self.X = derive_block(seed, TAG_X, self.N, m, p)
        self.D1 = derive_diag(seed, TAG_D1, self.N, p)
        self.D2 = derive_diag(seed, TAG_D2, self.M, p)


def blackbox_apply(A, p: int, side: int, d1: np.ndarray, d2: np.ndarray, v: np.ndarray) -> np.ndarray:
    v = _c(v, np.uint32).copy()
    N = v.shape[0]
    w = v.shape[1] if v.ndim == 2 else 1
    rp, ci, va = _csr_args(A)
    d1 = _c(d1, np.uint32)
    d2 = _c(d2, np.uint32)
    load().or_blackbox_apply(A.rows, A.cols, _p(rp), _p(ci), _p(va), p, side, _p(d1), _p(d2), w, _p(v))
    return v.reshape(N, w)


def blackbox_apply_rows(A, p: int, side: int, d1: np.ndarray, d2: np.ndarray, v: np.ndarray,
                        rows) -> np.ndarray:
    """Selected output rows of A~ v (Section 2.3's preconditioned black box),
    each computed on its own from the definition, for spot checks of full-size
    applications.  side 1 (N = rows): A~ = D1 A D2 A^T D1, so
    (A~ v)[x] = d1[x] sum_{y in row x of A} A[x,y] d2[y] sum_{z in col y} A[z,y] d1[z] v[z];
    side 0 (N = cols): the same with A^T in place of A.  Plain numpy, one
    residue product reduced mod p at a time."""
    v = np.asarray(v, dtype=np.uint64)
    if v.ndim == 1:
        v = v[:, None]
    d1 = np.asarray(d1, dtype=np.uint64)
    d2 = np.asarray(d2, dtype=np.uint64)
    rp = np.asarray(A.rowptr, dtype=np.int64)
    ci = np.asarray(A.colidx, dtype=np.int64)
    va = np.asarray(A.vals, dtype=np.int64)
    ri = np.repeat(np.arange(A.rows, dtype=np.int64), np.diff(rp))
    order = np.argsort(ci, kind="stable")  # column-major view of A
    cp = np.zeros(A.cols + 1, dtype=np.int64)
    np.add.at(cp, ci + 1, 1)
    cp = np.cumsum(cp)
    c_rows, c_vals = ri[order], va[order]

    def row_of_A(x):
        return ci[rp[x]:rp[x + 1]], va[rp[x]:rp[x + 1]]

    def col_of_A(y):
        return c_rows[cp[y]:cp[y + 1]], c_vals[cp[y]:cp[y + 1]]

    # M = A (side 1) or A^T (side 0): rows of M and columns of M
    m_row, m_col = (row_of_A, col_of_A) if side == 1 else (col_of_A, row_of_A)
    P = np.uint64(p)
    out = np.zeros((len(rows), v.shape[1]), dtype=np.uint64)
    for k, x in enumerate(rows):
        ys, ay = m_row(int(x))
        acc = np.zeros(v.shape[1], dtype=np.uint64)
        for y, a in zip(ys, ay):
            zs, az = m_col(int(y))
            u = np.zeros(v.shape[1], dtype=np.uint64)
            for z, b in zip(zs, az):
                t = (d1[z] * v[z]) % P                          # d1[z] v[z]
                u = (u + (np.uint64(int(b) % p) * t) % P) % P   # + A[z,y] d1[z] v[z]
            w = (d2[y] * u) % P
            acc = (acc + (np.uint64(int(a) % p) * w) % P) % P
        out[k] = (d1[x] * acc) % P
    return out.astype(np.uint32)


def sequence(A, setup: Setup, L: Optional[int] = None, return_last: bool = False):
    """S (L x m x n) with S_i = X^T A~^i Y mod p."""
    L = seq_length(setup.N, setup.m, setup.n) if L is None else L
    S = np.empty((L, setup.m, setup.n), dtype=np.uint32)
    V = np.empty((setup.N, setup.n), dtype=np.uint32)
    rp, ci, va = _csr_args(A)
    load().or_sequence(A.rows, A.cols, _p(rp), _p(ci), _p(va), setup.p, setup.side,
                       _p(setup.D1), _p(setup.D2), setup.m, setup.n, _p(_c(setup.X, np.uint32)),
                       _p(_c(setup.Y, np.uint32)), L, _p(S), _p(V))
    return (S, V) if return_last else S


def project(X: np.ndarray, V: np.ndarray, p: int) -> np.ndarray:
    X = _c(X, np.uint32)
    V = _c(V, np.uint32)
    N, m = X.shape
    n = V.shape[1]
    S = np.empty((m, n), dtype=np.uint32)
    load().or_project(N, m, n, _p(X), _p(V), p, _p(S))
    return S


# ---------------------------------------------------------------------------
# rank by elimination
# ---------------------------------------------------------------------------

def rank_dense(a: np.ndarray, p: int) -> int:
    a = np.array(a, dtype=np.int64, copy=True, order="C")
    if a.size == 0:
        return 0
    return int(load().or_rank_dense(a.shape[0], a.shape[1], _p(a), p))


def det_dense(a: np.ndarray, p: int) -> int:
    a = np.array(np.asarray(a, dtype=np.int64) % p, dtype=np.uint64, order="C")
    return int(load().or_det_dense(a.shape[0], _p(a), p))


def rank_sparse(A, p: int) -> int:
    rp, ci, va = _csr_args(A)
    return int(load().or_rank_sparse(A.rows, A.cols, _p(rp), _p(ci), _p(va), p))


# ---------------------------------------------------------------------------
# generators
# ---------------------------------------------------------------------------

def berlekamp_massey(s: np.ndarray, p: int):
    """Returns (Lc, f) with f the monic minimal polynomial of the scalar
    sequence, f[k] = coefficient of x^k: sum_k f[k] s[i + k] = 0."""
    s = _c(s, np.uint32).ravel()
    conn = np.zeros(len(s) + 1, dtype=np.uint32)
    Lc = int(load().or_berlekamp_massey(_p(s), len(s), p, _p(conn)))
    f = np.zeros(Lc + 1, dtype=np.uint64)
    for j in range(Lc + 1):  # f(x) = x^Lc conn(1/x)
        f[Lc - j] = conn[j]
    return Lc, f


def mbasis(S: np.ndarray, p: int, Dcap: Optional[int] = None):
    """Order-L sigma-basis of [S(x) | -I_m] with shift (0^n, 1^m).
    Returns (M [D+1, q, q] uint32, deg [q] int32)."""
    S = _c(S, np.uint32)
    L, m, n = S.shape
    q = m + n
    Dcap = L + 1 if Dcap is None else Dcap
    M = np.zeros((Dcap + 1, q, q), dtype=np.uint32)
    deg = np.zeros(q, dtype=np.int32)
    rc = load().or_mbasis(_p(S), L, m, n, p, Dcap, _p(M), _p(deg))
    if rc != 0:
        raise RuntimeError("mbasis: degree cap exceeded")
    return M[: int(deg.max()) + 1].copy(), deg


def select_generator(M: np.ndarray, deg: np.ndarray, n: int):
    """The n columns of least shifted degree (ties by index) give [P; Q];
    F_j(x) = x^{delta_j} P_j(1/x).  Returns (cols, delta, P, F) with
    P, F as [D+1, n, n] coefficient arrays."""
    q = M.shape[1]
    cols = sorted(range(q), key=lambda c: (int(deg[c]), c))[:n]
    delta = np.array([int(deg[c]) for c in cols], dtype=np.int64)
    D = int(delta.max()) if n else 0
    P = np.zeros((D + 1, n, n), dtype=np.uint32)
    F = np.zeros((D + 1, n, n), dtype=np.uint32)
    for j, c in enumerate(cols):
        dj = int(delta[j])
        top = min(dj, M.shape[0] - 1)
        P[: top + 1, :, j] = M[: top + 1, :n, c]
        for k in range(dj + 1):
            t = dj - k
            if t < M.shape[0]:
                F[k, :, j] = M[t, :n, c]
    return cols, delta, P, F


def det_valuation(G: np.ndarray, p: int, T0: int = 4) -> Optional[int]:
    """x-adic valuation of det G (G: [D+1, n, n]); None if det G = 0."""
    G = _c(G, np.uint32)
    D1, n, _ = G.shape
    if n == 0:
        return 0
    T = max(T0, 2)
    limit = 2 * (D1 * n + 2)
    while True:
        Tp = min(T, D1 + T)  # coefficients beyond D are zero
        GT = np.zeros((Tp, n, n), dtype=np.uint32)
        k = min(Tp, D1)
        GT[:k] = G[:k]
        v = int(load().or_det_valuation(_p(GT), n, Tp, p))
        if v >= 0:
            return v
        if T > limit:
            return None
        T *= 2


def det_poly(G: np.ndarray, p: int) -> np.ndarray:
    """det G as a polynomial, by evaluation at n*D+1 points and Lagrange
    interpolation (the paper's evaluation/interpolation fallback, Section 2.5).
    Tiny inputs only."""
    G = _c(G, np.uint32)
    D1, n, _ = G.shape
    D = D1 - 1
    npts = n * D + 1
    assert npts < p
    xs = list(range(1, npts + 1))
    ys = [int(load().or_det_poly_eval(_p(G), n, D, x, p)) for x in xs]
    # Lagrange interpolation, coefficients low -> high
    coef = [0] * npts
    for i, xi in enumerate(xs):
        num = [1]
        den = 1
        for j, xj in enumerate(xs):
            if j == i:
                continue
            num = [(a - xj * b) % p for a, b in zip([0] + num, num + [0])]
            den = den * (xi - xj) % p
        f = ys[i] * pow(den, p - 2, p) % p
        for k in range(len(num)):
            coef[k] = (coef[k] + f * num[k]) % p
    return np.array(coef, dtype=np.int64)


def rank_readout(M: np.ndarray, deg: np.ndarray, n: int, p: int) -> dict:
    """Section 2.5 step 4: r = deg det F - codeg det F.  With
    F_j(x) = x^{delta_j} P_j(1/x):  deg det F = sum delta - v_x(det P) and
    codeg det F = v_x(det F).  (When P(0) is nonsingular F is column reduced
    and deg det F is the sum of its column degrees -- the paper's Popov
    shortcut.)"""
    cols, delta, P, F = select_generator(M, deg, n)
    vP = det_valuation(P, p)
    vF = det_valuation(F, p)
    if vP is None or vF is None:
        raise RuntimeError("singular generator")
    sd = int(delta.sum())
    deg_det = sd - vP
    return dict(rank=deg_det - vF, deg_det=deg_det, codeg=vF, sum_delta=sd, vP=vP,
                cols=cols, delta=delta, F=F, P=P)


def early_termination_point(S: np.ndarray, p: int, chunk: int, quiet: int) -> Optional[int]:
    """Early termination (Section 4 mentions it; Table tab:r-time's 2 + 2r/p
    iterations say how many terms the rank needs; no criterion is given).
    Reading: the orders are taken in chunks of `chunk`; before the chunk
    [k0, k0 + b), the generator candidates are the n columns of least
    (shifted degree, index) of the order-k0 sigma-basis of [S | -I_m]; the
    chunk is quiet when every candidate has shifted degree <= k0 and zero
    residual [S(x) | -I_m] col mod p at every order of the chunk.  Quiet
    orders are counted over consecutive quiet chunks.  Returns the order count
    k0 + b at which the count first reaches `quiet` (the generator is then
    taken as final), or None if it never does within the L terms of S."""
    S = _c(S, np.uint32)
    L, m, n = S.shape
    q = m + n
    So = S.astype(object)
    count = 0
    for k0 in range(0, L, chunk):
        b = min(chunk, L - k0)
        if k0 == 0:
            M = np.zeros((1, q, q), dtype=np.uint32)
            for c in range(q):
                M[0, c, c] = 1
            deg = np.array([0] * n + [1] * m, dtype=np.int32)
        else:
            M, deg = mbasis(S[:k0], p)
        cand = sorted(range(q), key=lambda c: (int(deg[c]), c))[:n]
        quiet_chunk = all(int(deg[c]) <= k0 for c in cand)
        if quiet_chunk:
            Mo = M.astype(object)
            for c in cand:
                for k in range(k0, k0 + b):
                    # order-k coefficient of S(x) P_c(x) - Q_c(x)
                    r = np.zeros(m, dtype=object)
                    for t in range(min(k, Mo.shape[0] - 1) + 1):
                        r = r + So[k - t].dot(Mo[t, :n, c])
                    if k < Mo.shape[0]:
                        r = r - Mo[k, n:, c]
                    if any(int(v) % p for v in r):
                        quiet_chunk = False
                        break
                if not quiet_chunk:
                    break
        count = count + b if quiet_chunk else 0
        if count >= quiet:
            return k0 + b
    return None


def rank_wiedemann(A, p: int, m: int, n: int, seed: int, side: Optional[int] = None,
                   symmetric: bool = False, L: Optional[int] = None) -> dict:
    """The paper's block Wiedemann rank algorithm (Section 2.5, steps 1-4)."""
    st = Setup(A, p, m, n, seed, side, symmetric)
    if st.N == 0:
        return dict(rank=0, S=np.zeros((0, m, n), np.uint32))
    S = sequence(A, st, L)
    M, deg = mbasis(S, p)
    out = rank_readout(M, deg, n, p)
    out.update(S=S, M=M, deg=deg, setup=st)
    return out


# ---------------------------------------------------------------------------
# polynomial matrix helpers for checks (plain numpy with Python ints)
# ---------------------------------------------------------------------------

def polymat_mul(A: np.ndarray, B: np.ndarray, p: int, trunc: Optional[int] = None) -> np.ndarray:
    """C(x) = A(x) B(x) mod p, coefficient arrays [deg+1, r, c]."""
    da, db = A.shape[0], B.shape[0]
    dc = da + db - 1 if trunc is None else min(trunc, da + db - 1)
    C = np.zeros((dc, A.shape[1], B.shape[2]), dtype=object)
    Ao = A.astype(object)
    Bo = B.astype(object)
    for i in range(da):
        for j in range(db):
            if i + j < dc:
                C[i + j] = C[i + j] + Ao[i].dot(Bo[j])
    return (C % p).astype(np.int64)
