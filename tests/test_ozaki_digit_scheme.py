"""The digit scheme of the FP64-accurate tensor-core products, emulated on the
CPU in numpy (no GPU, no oracle): the claims the kernel's design rests on.

A row with max |x| < 2^(e-1) is scaled by 2^(bS - e), rounded to an integer
and written as S balanced base-2^b digits |d| <= 2^(b-1); slice pair (t, u)
contributes sum_k d_t d_u 2^(-b(t+u+2)) 2^(e_i+f_j), and the pairs with
t + u <= S - 1 are kept.  Checked for the three widths the library uses
(b = 6, S = 9; b = 7, S = 8; b = 8, S = 7):

* the digits are exact BF16 values and rebuild the rounded integer;
* at the largest inner dimension each width is used for (2^(26 - 2b)), a
  pair's sum over K stays within 2^24 even for the worst digits, so the
  FP32 accumulation is exact;
* a product Y = A B^H built this way errs by well under 16 sqrt(K) 2^-53 of
  the operand scales (the GPU test's tight bound), against an extended-
  precision reference, and leaving out the top level (t + u = S - 1) pushes
  it far above that bound.
"""
import numpy as np
import pytest

WIDTHS = [(6, 9), (7, 8), (8, 7)]


def _digits(x, b, S):
    """Row exponents and the S balanced digits (t = 0 most significant)."""
    m = np.max(np.abs(x), axis=1)
    _, ex = np.frexp(m)                      # m = f 2^ex, f in [0.5, 1)
    e = np.where(m > 0, ex + 1, -100000)     # max |x| < 2^(e - 1)
    v = np.rint(np.ldexp(x, (b * S - e)[:, None])).astype(np.int64)
    assert np.all(np.abs(v) < 2 ** (b * S - 1))
    half, mask = 1 << (b - 1), (1 << b) - 1
    d = np.zeros((S,) + x.shape, dtype=np.int64)
    for t in range(S - 1, 0, -1):
        d[t] = ((v + half) & mask) - half
        v = (v - d[t]) >> b
    d[0] = v
    return d, e


def _bf16_exact(d):
    """An integer is exact in BF16 if it has at most 8 significant bits."""
    a = np.abs(d)
    a = a[a > 0]
    while a.size and np.any(a % 2 == 0):
        a = np.where(a % 2 == 0, a // 2, a)
    return bool(np.all(a < 256))


def _product(A, B, b, S, drop_top=False):
    """Y = A B^H from the digit slices of A's and B's planes (complex)."""
    (dAr, eA), (dAi, _) = _digits_pair(A, b, S)
    (dBr, eB), (dBi, _) = _digits_pair(B, b, S)
    N = A.shape[0]
    top = S - 1 - (1 if drop_top else 0)
    acc_r = np.zeros((N, N), dtype=object)
    acc_i = np.zeros((N, N), dtype=object)
    for t in range(S):
        for u in range(S - t):
            if t + u > top:
                continue
            f = lambda z: z.astype(np.float64)
            rr = f(dAr[t]) @ f(dBr[u]).T          # exact: integers below 2^53
            ii = f(dAi[t]) @ f(dBi[u]).T
            ri = f(dAr[t]) @ f(dBi[u]).T
            ir = f(dAi[t]) @ f(dBr[u]).T
            w = 1 << (b * (S - 1 - (t + u)))        # common unit 2^(-b(S+1))
            acc_r = acc_r + (rr + ii).astype(np.int64).astype(object) * w
            acc_i = acc_i + (ir - ri).astype(np.int64).astype(object) * w
    unit = (eA[:, None] + eB[None, :]) - b * (S + 1)
    to_f = np.vectorize(lambda q, s: float(np.ldexp(float(q), int(s))), otypes=[np.float64])
    return to_f(acc_r, unit) + 1j * to_f(acc_i, unit)


def _digits_pair(A, b, S):
    """Digits of the real and imaginary planes with one exponent per row over both."""
    both = np.concatenate([A.real, A.imag], axis=1)
    d, e = _digits(both, b, S)
    n = A.shape[1]
    return (d[:, :, :n], e), (d[:, :, n:], e)


@pytest.mark.parametrize("b,S", WIDTHS)
def test_digits_are_exact_and_rebuild_the_integer(b, S):
    rng = np.random.default_rng(b)
    x = rng.standard_normal((64, 64)) * np.exp(rng.uniform(-30, 30, size=(64, 1)))
    d, e = _digits(x, b, S)
    assert np.all(np.abs(d) <= 1 << (b - 1))
    assert _bf16_exact(d)
    v = sum(d[t] * (1 << (b * (S - 1 - t))) for t in range(S))
    assert np.array_equal(v, np.rint(np.ldexp(x, (b * S - e)[:, None])).astype(np.int64))


@pytest.mark.parametrize("b,S", WIDTHS)
def test_pair_sums_stay_exact_in_fp32_at_the_largest_k(b, S):
    K = 1 << (26 - 2 * b)                     # 16384, 4096, 1024
    worst = (1 << (b - 1)) ** 2 * K            # every product at its largest
    assert worst <= 1 << 24
    # the extreme integers a row can produce still give digits within 2^(b-1)
    lim = (1 << (b * S - 1)) - 1
    x = np.ldexp(np.array([[float(lim), -float(lim), 1.0]]), -(b * S) + 1)
    d, _ = _digits(x, b, S)
    assert np.max(np.abs(d)) <= 1 << (b - 1)


@pytest.mark.parametrize("b,S", WIDTHS)
def test_product_error_and_top_level_sensitivity(b, S):
    N = 128
    rng = np.random.default_rng(10 + b)
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    B = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    A /= np.max(np.abs(A))
    B /= np.max(np.abs(B))
    Al = (A.real.astype(np.longdouble), A.imag.astype(np.longdouble))
    Bl = (B.real.astype(np.longdouble), B.imag.astype(np.longdouble))
    ref_r = Al[0] @ Bl[0].T + Al[1] @ Bl[1].T
    ref_i = Al[1] @ Bl[0].T - Al[0] @ Bl[1].T
    bound = 16 * np.sqrt(N) * 2.0 ** -53

    def err(Y):
        return float(max(np.max(np.abs(Y.real - ref_r)), np.max(np.abs(Y.imag - ref_i))))

    full = err(_product(A, B, b, S))
    dropped = err(_product(A, B, b, S, drop_top=True))
    assert full < 0.3 * bound          # 0.04-0.2 of the bound in practice
    assert dropped > 3 * bound         # 5-16 times the bound
