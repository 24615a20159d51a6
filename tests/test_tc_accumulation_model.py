"""Accumulation model of the tensor-core MMA, and the exact-slice plan for
the double-float contractions of the evaluation (kinematics F = U + B q and
residual r = B^T (w P), Sec. 3.2.1, Eqs. ROM_assumption and ROMintforce).

Model.  One MMA k-step adds K exact products to the float32 accumulator the
way the tensor core was measured to: the products and the accumulator are
aligned to the largest exponent among them, each keeps the `bits` bits below
that exponent (the rest is truncated toward zero), the aligned terms are
summed exactly and the sum is truncated to a `bits`-bit significand.  This
model reproduces the measured error tail of the tf32 kernels, where the
products added to an accumulator that already holds a partial sum lose
their low bits; rounding to nearest does not.

Exact slicing (the Ozaki scheme).  Each operand is scaled by a power of two
per row (A) or per column (B) and cut into L digits of s bits:
    A = sa * sum_l dA_l 2^-s(l+1),   |dA_l| < 2^s, dA_l integer,
so the product is a sum over shift levels t = l1 + l2 of integer matrices
    P_t = sum_(l1 + l2 = t) dA_l1 dB_l2,
each computed by MMAs on small-integer operands (exact in bf16 for s <= 8).
While K * (pairs in the level) * 2^(2s) stays below 2^bits, every partial
sum is an integer below 2^bits: the aligned truncation of the model finds no
bit below the quantum to drop, and the level sums are exact.  The levels are
combined on the CUDA cores; levels t >= T are dropped.

The tests pin the model on cases with known answers, then check, on the
residual's shape (32 points, 200 ECM points x 4 stress components, 24
modes; rows scaled over three decades), that 5-bit digits on 10 levels give
exact level sums for a 22-, 23- or 24-bit accumulator and a result within
the truncation bound of the exact product, while 6-bit digits overflow the
accumulator on worst-case operands.
"""
import math

import numpy as np
import pytest


# ---------------------------------------------------------------- the model
def _floor_log2(x):
    # floor(log2 |x|) for x != 0 (0 where x == 0)
    m, e = np.frexp(np.abs(x))
    return np.where(x != 0, e - 1, 0)


def mma_step(acc, prods, bits=24):
    """acc (R,), prods (R, K) exact products (float64) -> accumulator after
    one k-step under the aligned-truncation model."""
    terms = np.concatenate([acc[:, None], prods], axis=1)
    e = _floor_log2(np.abs(terms).max(axis=1))
    q = np.ldexp(1.0, e - bits + 1)[:, None]
    s = (np.trunc(terms / q) * q).sum(axis=1)  # exact: < 2^(bits + 5) quanta
    qs = np.ldexp(1.0, _floor_log2(s) - bits + 1)
    return np.where(s != 0, np.trunc(s / qs) * qs, 0.0)


def mma(Ad, Bd, ksz, bits=24, acc=None):
    """C = A B through k-steps of ksz under the model; A (M, K), B (K, N)
    with products exact in float64 (small integers here)."""
    M, K = Ad.shape
    N = Bd.shape[1]
    acc = np.zeros(M * N) if acc is None else acc
    for k0 in range(0, K, ksz):
        a = Ad[:, k0:k0 + ksz]
        b = Bd[k0:k0 + ksz, :]
        prods = (a[:, None, :] * b.T[None, :, :]).reshape(M * N, -1)
        acc = mma_step(acc, prods, bits)
    return acc.reshape(M, N)


# ------------------------------------------------------------- the slicing
def slice_rows(X, s, L):
    """X (R, K) -> power-of-two row scales sa (R,) and digits (L, R, K),
    integers with |d| < 2^s, X = sa * sum_l d_l 2^-s(l+1) + remainder."""
    mx = np.abs(X).max(axis=1)
    sa = np.ldexp(1.0, np.frexp(mx)[1])  # |X / sa| < 1
    Y = X / sa[:, None]
    digits = []
    for _ in range(L):
        Y = Y * 2.0 ** s
        d = np.trunc(Y)
        digits.append(d)
        Y = Y - d
    return sa, np.array(digits)


def sliced_levels(A, B, s, L, T, ksz, bits):
    """Level sums P_t (t < T) of the sliced product through the model, with
    the exact integer level sums beside them."""
    sa, dA = slice_rows(A, s, L)
    sb, dBt = slice_rows(B.T, s, L)
    dB = np.transpose(dBt, (0, 2, 1))
    model, exact = [], []
    for t in range(T):
        acc = None
        ex = np.zeros((A.shape[0], B.shape[1]), dtype=object)
        for l1 in range(max(0, t - L + 1), min(t, L - 1) + 1):
            l2 = t - l1
            acc = mma(dA[l1], dB[l2], ksz, bits, None if acc is None else acc.reshape(-1))
            ex = ex + np.dot(dA[l1].astype(np.int64).astype(object), dB[l2].astype(np.int64).astype(object))
        model.append(acc)
        exact.append(ex)
    return sa, sb, model, exact


def exact_product(A, B):
    """A B exactly, as Python integers over a common power of two."""
    ea = int(-np.frexp(np.abs(A[A != 0])).__getitem__(1).min()) + 60
    eb = int(-np.frexp(np.abs(B[B != 0])).__getitem__(1).min()) + 60
    Ai = np.vectorize(lambda x: int(math.ldexp(x, ea)), otypes=[object])(A)
    Bi = np.vectorize(lambda x: int(math.ldexp(x, eb)), otypes=[object])(B)
    return np.dot(Ai, Bi), ea + eb


def residual_operands(seed, P=32, M=200, G=4, n=24, decades=3.0):
    """w P (points x (ECM point, component)), rows scaled over `decades`,
    and B (ECM point rows x modes) of the residual r = B^T (w P)."""
    g = np.random.default_rng(seed)
    wP = g.standard_normal((P, M * G)) * 10.0 ** g.uniform(-decades, 0.0, (P, 1))
    B = g.standard_normal((M * G, n)) * 10.0 ** g.uniform(-1.0, 1.0, (1, n))
    return wP, B


# ---------------------------------------------------------------- pins
def test_model_single_product_truncates_toward_zero():
    g = np.random.default_rng(0)
    x = g.standard_normal(2000) * 10.0 ** g.uniform(-5, 5, 2000)
    r = mma_step(np.zeros(2000), x[:, None])
    assert np.all(r.astype(np.float32).astype(np.float64) == r)  # a float32 value
    assert np.all(np.abs(r) <= np.abs(x)) and np.all(np.sign(r) == np.sign(x))
    ulp = np.ldexp(1.0, _floor_log2(x) - 23)
    assert np.all(np.abs(x) - np.abs(r) < ulp)
    # round to nearest would differ on about half of them
    assert np.mean(r != x.astype(np.float32).astype(np.float64)) > 0.3


def test_model_drops_small_products_against_a_large_accumulator():
    # 8 products of 2^-25 onto 1.0: each is below the quantum 2^-23 of the
    # aligned terms and vanishes, although 1 + 2^-22 is a float32 value
    r = mma_step(np.array([1.0]), np.full((1, 8), 2.0 ** -25))
    assert r[0] == 1.0
    # alone, the same products sum exactly
    assert mma_step(np.array([0.0]), np.full((1, 8), 2.0 ** -25))[0] == 2.0 ** -22
    # with 8 products of 2^-23 every one survives
    assert mma_step(np.array([1.0]), np.full((1, 8), 2.0 ** -23))[0] == 1.0 + 2.0 ** -20


def test_model_is_exact_on_integer_sums_below_the_significand():
    g = np.random.default_rng(1)
    A = g.integers(-31, 32, (16, 800)).astype(np.float64)
    B = g.integers(-31, 32, (800, 8)).astype(np.float64)
    C = mma(A, B, 16)
    assert np.array_equal(C, A @ B)  # |partial sums| < 800 * 31^2 < 2^24
    # the same through 8-wide tf32 k-steps
    assert np.array_equal(mma(A, B, 8), A @ B)


def test_slicing_reconstructs_the_operand():
    g = np.random.default_rng(2)
    X = g.standard_normal((8, 50)) * 10.0 ** g.uniform(-3, 3, (8, 1))
    for s, L in ((5, 10), (8, 6)):
        sa, d = slice_rows(X, s, L)
        assert np.all(np.abs(d) < 2 ** s) and np.array_equal(d, np.trunc(d))
        rec = sa[:, None] * sum(d[l] * 2.0 ** (-s * (l + 1)) for l in range(L))
        assert np.all(np.abs(rec - X) <= sa[:, None] * 2.0 ** (-s * L))


# ------------------------------------------------ the residual's contraction
@pytest.mark.parametrize('bits', [24, 23, 22])
def test_exact_slices_reproduce_the_residual_contraction(bits):
    s, L, T, ksz = 5, 10, 10, 16  # 5-bit digits in bf16, k-steps of 16
    wP, B = residual_operands(3)
    K = wP.shape[1]
    sa, sb, model, exact = sliced_levels(wP, B, s, L, T, ksz, bits)
    # level t has t + 1 digit pairs: K (t + 1) 2^(2s) <= 2^bits for every
    # level when 2s + log2 K + log2 T <= bits (23.0 bits here); random signs
    # keep the sums far lower, so a 22-bit accumulator is exact as well
    for t in range(T):
        assert np.array_equal(model[t].astype(np.int64).astype(object), exact[t]), t
    assert 2 * s + math.log2(K) + math.log2(T) <= 23.0
    # the levels of the model, combined exactly, against the exact product
    comb = sum(model[t].astype(np.int64).astype(object) * (1 << (s * (T - t))) for t in range(T))
    Cx, ex = exact_product(wP, B)
    P_, N_ = wP.shape[0], B.shape[1]
    Cs = np.array([[math.ldexp(float(comb[i, j]), -s * (T + 2)) * sa[i] * sb[j] for j in range(N_)]
                   for i in range(P_)])
    Ce = np.array([[math.ldexp(float(Cx[i, j]), -ex) for j in range(N_)] for i in range(P_)])
    # bound: dropped levels t >= T (t + 1 pairs below 2^-st each) and the
    # digit remainders (below 2^-sL each), per term, relative to sa sb
    per_term = sum((t + 1) * 2.0 ** (-s * t) for t in range(T, 2 * L)) + 2 * 2.0 ** (-s * L)
    err = np.abs(Cs - Ce) / np.outer(sa, sb)
    assert err.max() <= K * per_term
    # relative to |wP| |B|: within double-float accuracy (2^-44; the
    # dropped levels give about 1.2e-14 here, a float64 contraction 3e-16)
    ab = np.abs(wP) @ np.abs(B)
    rel = (np.abs(Cs - Ce) / ab).max()
    assert rel <= 2.0 ** -44, rel


def test_six_bit_digits_overflow_the_accumulator_on_worst_case_operands():
    # all digits maximal and of one sign: the level sums reach
    # K * pairs * (2^s - 1)^2, below 2^24 for s = 5 (800 * 10 * 31^2 = 7.7e6),
    # above it for s = 6 (800 * 8 * 63^2 = 2.5e7)
    K, n = 800, 4
    for s, L, ok in ((5, 10, True), (6, 8, False)):
        v = 1.0 - 2.0 ** (-s * L)  # every digit 2^s - 1 (exact in float64)
        A = np.full((2, K), v)
        Bm = np.full((K, n), v)
        sa, sb, model, exact = sliced_levels(A, Bm, s, L, L, 16, 24)
        assert sa[0] == 1.0 and np.all(slice_rows(A, s, L)[1] == 2 ** s - 1)
        same = all(np.array_equal(model[t].astype(np.int64).astype(object), exact[t]) for t in range(L))
        assert same == ok, s
