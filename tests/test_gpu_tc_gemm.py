"""Tensor-core digit-plane GEMM (the mixed-precision RI-K engine, Eqs. k_ri_2
and tp) against an FP64 product.

Bound: with s digits every operand element keeps 7 + 8 (s - 1) bits below the
largest exponent of its row's K block, and the dropped digit pairs weigh less
than 2^{-8s} of the leading term, so
    |C - A B^T| <= c 2^{-(7 + 8(s-1))} K max|A_row| max|B_row|
with a small constant c (8 here, covering both sources and the final rounding).
"""
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


@pytest.mark.parametrize("M,N,K", [(300, 70, 200), (128, 40, 192), (257, 16, 64), (33, 129, 1000), (64, 33, 31)])
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
