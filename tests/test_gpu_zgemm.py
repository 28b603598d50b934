"""hbs_zgemm in its three arithmetics against numpy's FP64 product: FP64 (DFMA), double-float
(float pairs on the FP32 pipes) and tensor (bf16 digit planes on the tcgen05 tensor cores,
exact FP32 accumulation, double-float recombination).  Errors are measured per entry against
k max|a| max|b| (the scale of every bound here) and, for rows of very different size, against
the row's own scale."""
import numpy as np
import pytest

from gpu_util import dev, require_lib

pytestmark = pytest.mark.gpu


def _cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _run(hbs, m, n, k, alpha, beta, trans_a, prec, A, B, C0):
    import torch
    a = dev(np.asfortranarray(A).ravel(order="F"))
    b = dev(np.asfortranarray(B).ravel(order="F"))
    c = dev(np.asfortranarray(C0).ravel(order="F"))
    lda = A.shape[0]
    hbs.zgemm(m, n, k, alpha, a, lda, trans_a, b, k, beta, c, m, prec)
    torch.cuda.synchronize()
    return c.cpu().numpy().reshape((n, m)).T


CASES = [  # m, n, k, trans_a
    (300, 70, 5000, 0),
    (129, 33, 4100, 1),   # one row past a 128-row tile, k not a multiple of 64
    (700, 190, 16384, 0),  # several k splits
]


@pytest.mark.parametrize("m,n,k,trans_a", CASES)
def test_zgemm_three_arithmetics(m, n, k, trans_a):
    hbs = require_lib()
    rng = np.random.default_rng(m + n + k)
    A = _cplx(rng, k, m) if trans_a else _cplx(rng, m, k)
    B = _cplx(rng, k, n)
    C0 = _cplx(rng, m, n)
    alpha, beta = 0.7 - 0.2j, 0.3 + 0.1j
    opA = A.T if trans_a else A
    ref = alpha * (opA @ B) + beta * C0
    scale = k * np.abs(A).max() * np.abs(B).max()
    for prec, bound in ((hbs.PRECISION_FP64, 1e-15), (hbs.PRECISION_DOUBLE_FLOAT, 1e-14),
                        (hbs.PRECISION_TENSOR, 1e-14)):
        got = _run(hbs, m, n, k, alpha, beta, trans_a, prec, A, B, C0)
        err = np.abs(got - ref).max() / scale
        assert err < bound, (prec, err)


def test_zgemm_tensor_rows_of_different_size():
    """Each row of op(A) and column of B has its own power-of-two scale, so a row 1e-9 times
    smaller than the others keeps its relative accuracy."""
    hbs = require_lib()
    rng = np.random.default_rng(3)
    m, n, k = 256, 40, 8192
    A = _cplx(rng, m, k)
    A[::7] *= 1e-9
    B = _cplx(rng, k, n)
    B[:, ::5] *= 1e6
    ref = A @ B
    got = _run(hbs, m, n, k, 1.0, 0.0, 0, hbs.PRECISION_TENSOR, A, B, np.zeros((m, n), complex))
    rs = k * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]
    assert (np.abs(got - ref) / rs).max() < 1e-14


def test_zgemm_tensor_exact_on_digit_grids():
    """Integer operands below 2^7 are single digits: the tensor product is exact."""
    hbs = require_lib()
    rng = np.random.default_rng(4)
    m, n, k = 128, 32, 4096
    A = rng.integers(-127, 128, (m, k)) + 1j * rng.integers(-127, 128, (m, k))
    B = rng.integers(-127, 128, (k, n)) + 1j * rng.integers(-127, 128, (k, n))
    got = _run(hbs, m, n, k, 1.0, 0.0, 0, hbs.PRECISION_TENSOR, A.astype(complex), B.astype(complex),
               np.zeros((m, n), complex))
    assert np.array_equal(got, (A @ B).astype(complex))


def test_zgemm_rejects_bad_arguments():
    hbs = require_lib()
    import ctypes
    L = hbs.lib()
    one = (ctypes.c_double * 2)(1.0, 0.0)
    st = L.hbs_zgemm(4, 4, 4, one, None, 4, 0, None, 4, one, None, 4, 0, None)
    assert st == hbs.HBS_ERR_INVALID_ARG
    st = L.hbs_zgemm(4, 4, 4, one, ctypes.c_void_p(16), 2, 0, ctypes.c_void_p(16), 4, one, ctypes.c_void_p(16), 4, 0,
                     None)
    assert st == hbs.HBS_ERR_INVALID_ARG  # lda < m
    st = L.hbs_zgemm(4, 4, 4, one, ctypes.c_void_p(16), 4, 0, ctypes.c_void_p(16), 4, one, ctypes.c_void_p(16), 4, 7,
                     None)
    assert st == hbs.HBS_ERR_INVALID_ARG  # unknown precision
