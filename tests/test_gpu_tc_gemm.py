"""Tensor-core digit-plane GEMM (the mixed-precision RI-K engine, Eqs. k_ri_2
and tp) against an FP64 product.

Bound: with s digits every operand element keeps 7 + 8 (s - 1) bits below the
largest exponent of its row's K block, and the dropped digit pairs weigh less
than 2^{-8s} of the leading term, so
    |C - A B^T| <= c 2^{-(7 + 8(s-1))} K max|A_row| max|B_row|
with a small constant c (8 here, covering both sources and the final rounding).
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2407_19614_gb300 import rihf

pytestmark = pytest.mark.gpu


def _bound(A, B, digits, kblock):
    M, K = A.shape
    N = B.shape[0]
    bits = min(7 + 8 * (digits - 1), 55)
    kb = 32 * kblock if kblock else K
    bound = np.zeros((M, N))
    for k0 in range(0, K, kb):
        a = np.abs(A[:, k0:k0 + kb]).max(axis=1)
        b = np.abs(B[:, k0:k0 + kb]).max(axis=1)
        bound += min(kb, K - k0) * np.outer(a, b)
    return 8.0 * 2.0 ** (-bits) * bound + 4 * np.finfo(float).eps * (np.abs(A) @ np.abs(B).T)


def _case(M, N, K, seed, wide=False):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    if wide:   # rows spanning many orders of magnitude, plus exact zeros
        A *= 10.0 ** rng.uniform(-8, 8, size=(M, 1))
        B *= 10.0 ** rng.uniform(-8, 8, size=(N, 1))
        A[rng.random(A.shape) < 0.05] = 0.0
    return A, B


@pytest.mark.parametrize("M,N,K", [(300, 70, 200), (128, 40, 192), (257, 16, 64), (33, 129, 1000), (64, 33, 31),
                                   (20000, 100, 96)])
def test_tc_dgemm_seven_digits(M, N, K):
    A, B = _case(M, N, K, seed=M + N + K)
    C = rihf.tc_dgemm(A, B, digits=7)
    ref = A @ B.T
    err = np.abs(C - ref)
    assert np.all(err <= _bound(A, B, 7, 0)), err.max()
    # well above FP32 accuracy: relative to the natural scale sqrt(K)
    assert err.max() < 1e-12 * np.sqrt(K)


def test_tc_dgemm_wide_rows_and_blocks():
    A, B = _case(200, 96, 640, seed=3, wide=True)
    for kblock in (0, 1, 3):
        C = rihf.tc_dgemm(A, B, digits=7, kblock=kblock)
        err = np.abs(C - A @ B.T)
        assert np.all(err <= _bound(A, B, 7, kblock)), (kblock, (err / _bound(A, B, 7, kblock)).max())


@pytest.mark.parametrize("digits", [1, 2, 3, 4, 5, 6])
def test_tc_dgemm_fewer_digits(digits):
    A, B = _case(160, 48, 256, seed=digits)
    C = rihf.tc_dgemm(A, B, digits=digits)
    err = np.abs(C - A @ B.T)
    assert np.all(err <= _bound(A, B, digits, 0))
    if digits >= 2:   # each extra digit buys about 8 bits
        C1 = rihf.tc_dgemm(A, B, digits=digits - 1)
        assert err.max() < np.abs(C1 - A @ B.T).max() / 16


def test_tc_dgemm_small_integers_exact():
    # integer operands of at most 7 bits are single digits: the product is exact
    rng = np.random.default_rng(7)
    A = rng.integers(-100, 101, size=(130, 300)).astype(float)
    B = rng.integers(-100, 101, size=(20, 300)).astype(float)
    C = rihf.tc_dgemm(A, B, digits=7)
    assert np.array_equal(C, A @ B.T)


def test_tc_dgemm_rejects_bad_arguments():
    A = np.ones((4, 32 * 80))
    with pytest.raises(rihf.RihfError):
        rihf.tc_dgemm(A, A, digits=8)
    with pytest.raises(rihf.RihfError):   # 61 chunks per block would overflow the int64 sums
        rihf.tc_dgemm(A, A, digits=7, kblock=61)


def _value_of_digits(d):
    """The number in [1, 2) whose seven balanced base-256 digits (weights
    2^(48 - 8t) on the 2^-54 grid of its own exponent) are d."""
    V = sum(dt << (48 - 8 * t) for t, dt in enumerate(d))
    assert V % 4 == 0 and 2 ** 54 <= V < 2 ** 55
    return V / 2.0 ** 54          # exact: V / 4 has 53 bits


@pytest.mark.parametrize("digits,K", [(7, 1024), (5, 960)])
def test_tc_dgemm_accumulators_near_two_to_the_24(digits, K):
    """Digits close to +-127 with alternating signs make every product on an
    anti-diagonal of the digit pairs carry the same sign, so the FP32 TMEM sums
    between read-outs reach s * K' * 127^2 ~ 2^23.8 (K' = 32 floor(1024 / s / 32)
    elements: 128 for 7 digits, 192 for 5).  The result must equal, bit for
    bit, the integer replica of the digit-pair sums read out every K' elements
    (a white-box model of the read-out schedule: an FP32 sum that lost a bit
    changes it)."""
    dA = [127, -127, 127, -127, 127, -127, 124]
    dB = [127, -125, 123, -121, 119, -117, 116]
    xa, xb = _value_of_digits(dA), _value_of_digits(dB)
    M, N = 130, 40
    A = np.full((M, K), xa)
    B = np.full((N, K), xb)
    C = rihf.tc_dgemm(A, B, digits=digits)
    Kr = 32 * ((1024 // digits) // 32)
    S = 0
    for k0 in range(0, K, Kr):
        kk = min(Kr, K - k0)
        for g in range(2, digits + 2):
            v = kk * sum(dA[t - 1] * dB[g - t - 1] for t in range(1, g))
            assert abs(v) < 2 ** 24
            sh = 37 - 8 * (g - 2)
            S += v << sh if sh >= 0 else v >> -sh
    expect = float(Fraction(S, 2 ** 49))     # both exponents are those of [1, 2)
    assert np.all(C == expect), (C.min() - expect, C.max() - expect)
    bits = min(7 + 8 * (digits - 1), 55)
    assert abs(expect - K * xa * xb) <= 8 * 2.0 ** -bits * K * 4
