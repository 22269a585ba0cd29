"""The polynomial matrix product of PM-Basis (Section 2.4) through the C ABI
(three number-theoretic transforms and a Chinese remainder step) against the
oracle's product: full, truncated and middle products, element by element,
on shapes that span one and several transform tiles; at lengths the oracle's
quadratic loop cannot reach, the evaluation homomorphism C(x0) = A(x0) B(x0)
at random points and sampled coefficients from their defining sum; the
degenerate cases and the rejected arguments.  Integer work: every comparison
is exact."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wr():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0704_2351_gb300 import _build
    _build.build()
    from paper_0704_2351_gb300 import wr as w
    return w


@pytest.fixture(scope="module")
def ctx(wr):
    c = wr.wr_create(0)
    yield c
    wr.wr_destroy(c)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def from_dev(t):
    return t.cpu().numpy().view(np.uint32).astype(np.int64)


def gpu_product(wr, ctx, A, B, p, lo, hi):
    na, r, s = A.shape
    nb, _, t = B.shape
    C = torch.full((max(hi - lo, 1), r, t), -1, dtype=torch.int32, device="cuda")
    dA, dB = to_dev(A.reshape(-1)), to_dev(B.reshape(-1))
    torch.cuda.synchronize()  # the inputs are written before the context's stream reads them
    wr.wr_polymat_mul_device(ctx, p, dA, na, dB, nb, r, s, t, lo, hi, C)
    return from_dev(C)[:hi - lo]


def window(C, lo, hi):
    """Coefficients lo .. hi - 1 of the product whose coefficients are C (zero past them)."""
    out = np.zeros((hi - lo,) + C.shape[1:], dtype=np.int64)
    top = min(hi, C.shape[0])
    if top > lo:
        out[:top - lo] = C[lo:top]
    return out


PRIMES = [65521, 469762049, 1073741789, 2147483629, 2147483647]


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("na,nb,r,s,t", [(1, 1, 1, 1, 1), (5, 3, 2, 3, 4), (33, 65, 3, 5, 2), (130, 70, 4, 9, 8),
                                         (257, 129, 5, 2, 9), (700, 40, 2, 2, 2), (64, 64, 8, 16, 8)])
def test_product_equals_the_oracle(wr, ctx, p, na, nb, r, s, t):
    rng = np.random.default_rng(na * 7 + nb * 3 + r + p % 89)
    A = rng.integers(0, p, size=(na, r, s))
    B = rng.integers(0, p, size=(nb, s, t))
    full = na + nb - 1
    ref = oracle.polymat_mul(A, B, p)
    for lo, hi in [(0, full), (0, (full + 1) // 2), (na // 2, full), (nb // 3, na + nb // 2 if na > 1 else 1),
                   (full - 1, full + 5)]:
        lo, hi = min(lo, hi), max(lo, hi)
        assert np.array_equal(gpu_product(wr, ctx, A, B, p, lo, hi), window(ref, lo, hi)), (lo, hi)


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_residue_extremes(wr, ctx, p):
    """All entries p - 1 (the largest exact coefficients), ones, zeros and a mix."""
    na, nb, r, s, t = 90, 150, 3, 32, 4
    rng = np.random.default_rng(p % 1000)
    mix = np.array([0, 1, p - 1, p // 2, (p + 1) // 2, 255, 65536 % p], dtype=np.int64)
    for fa, fb in [(p - 1, p - 1), (1, 1), (0, p - 1), ("mix", "mix")]:
        A = rng.choice(mix, size=(na, r, s)) if fa == "mix" else np.full((na, r, s), fa, dtype=np.int64)
        B = rng.choice(mix, size=(nb, s, t)) if fb == "mix" else np.full((nb, s, t), fb, dtype=np.int64)
        full = na + nb - 1
        assert np.array_equal(gpu_product(wr, ctx, A, B, p, 0, full), oracle.polymat_mul(A, B, p))


def evaluate(P, x0, p):
    """P(x0) mod p for a long polynomial matrix: powers of x0 in blocks of 1024,
    products reduced one by one (below 2^62) and summed in uint64."""
    n, B = P.shape[0], 1024
    base = np.ones(B, dtype=np.uint64)
    for j in range(1, B):
        base[j] = int(base[j - 1]) * x0 % p
    X, f = pow(x0, B, p), 1
    pw = np.empty(-(-n // B) * B, dtype=np.uint64)
    for i in range(len(pw) // B):
        pw[i * B:(i + 1) * B] = base * np.uint64(f) % np.uint64(p)
        f = f * X % p
    terms = P.astype(np.uint64) * pw[:n, None, None] % np.uint64(p)
    return (terms.sum(axis=0) % np.uint64(p)).astype(object)


@pytest.mark.parametrize("na,nb,r,s,t", [(5000, 3300, 1, 1, 1), (70000, 1000, 2, 3, 2), (300001, 290000, 1, 2, 1),
                                         (9000, 9000, 4, 8, 4)])
def test_long_products_by_evaluation_and_sampled_coefficients(wr, ctx, na, nb, r, s, t):
    """Products whose transforms take two and three passes: C(x0) = A(x0) B(x0)
    mod p at random x0, and sampled coefficients C_k = sum_j A_j B_{k-j}."""
    p = 2147483629
    rng = np.random.default_rng(na + nb)
    A = rng.integers(0, p, size=(na, r, s))
    B = rng.integers(0, p, size=(nb, s, t))
    full = na + nb - 1
    C = gpu_product(wr, ctx, A, B, p, 0, full)
    for x0 in rng.integers(0, p, size=2):
        lhs = evaluate(C, int(x0), p)
        assert np.array_equal(lhs, evaluate(A, int(x0), p).dot(evaluate(B, int(x0), p)) % p)
    for k in list(rng.integers(0, full, size=6)) + [0, full - 1, na - 1, nb - 1]:
        j = np.arange(max(0, k - nb + 1), min(k, na - 1) + 1)
        prod = A[j][:, :, :, None].astype(np.uint64) * B[k - j][:, None, :, :].astype(np.uint64) % np.uint64(p)
        ck = prod.sum(axis=(0, 2)) % np.uint64(p)
        assert np.array_equal(C[k], ck.astype(np.int64)), k
    lo, hi = full // 3, full // 3 + 4097  # a middle window of the same product
    assert np.array_equal(gpu_product(wr, ctx, A, B, p, lo, hi), C[lo:hi])


def test_degenerate_cases(wr, ctx):
    p = 65521
    A = np.arange(12).reshape(2, 2, 3) % p
    B = np.arange(18).reshape(3, 3, 2) % p
    C = torch.full((4, 2, 2), -1, dtype=torch.int32, device="cuda")
    dA, dB = to_dev(A.reshape(-1)), to_dev(B.reshape(-1))
    torch.cuda.synchronize()
    wr.wr_polymat_mul_device(ctx, p, dA, 2, dB, 3, 2, 3, 2, 3, 3, C)
    assert (C == -1).all()  # an empty window writes nothing
    wr.wr_polymat_mul_device(ctx, p, dA, 0, dB, 3, 2, 3, 2, 0, 4, C)
    assert (C == 0).all()  # an empty factor gives the zero polynomial
    assert np.array_equal(gpu_product(wr, ctx, A, B, p, 4, 9), np.zeros((5, 2, 2), np.int64))  # past the product


def test_rejected_arguments(wr, ctx):
    d = torch.zeros(64, dtype=torch.int32, device="cuda")
    C = torch.zeros(64, dtype=torch.int32, device="cuda")
    for args in [(65521, 2, 2, 1, 1, 1, 3, 1), (65521, 2, 2, 0, 1, 1, 0, 2), (65521, 2, 2, 1, 1025, 1, 0, 2),
                 (65520, 2, 2, 1, 1, 1, 0, 2), (65521, -1, 2, 1, 1, 1, 0, 2)]:
        p, na, nb, r, s, t, lo, hi = args
        with pytest.raises(wr.WrError):
            wr.wr_polymat_mul_device(ctx, p, d, na, d, nb, r, s, t, lo, hi, C)
    # coefficients past the transform primes' product, and transforms longer
    # than 2^23 (buffers of the full sizes, so nothing is read out of range)
    p = 2147483647
    A = torch.zeros(400000 * 1024, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(wr.WrError):
        wr.wr_polymat_mul_device(ctx, p, A, 400000, A, 400000, 1, 1024, 1, 0, 8, C)
    del A
    A = torch.zeros((1 << 23) + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(wr.WrError):
        wr.wr_polymat_mul_device(ctx, p, A, (1 << 23) + 1, d, 2, 1, 1, 1, 0, 8, C)
