"""The oracle's threaded CSR products equal the sequential ones.

ThreadedCSR only shares rows among threads; each row is still one sequential
sum in storage order, so its products must equal scipy's CSR product to the
last bit whatever the thread count (the plain C loop is built without fused
multiply-adds), and the solvers must give the same iterates with it.
"""

import numpy as np
import pytest

from oracle import radon, spmv, tv
from paper_1705_07497_gb300 import inputs


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_products_equal_sequential_csr(threads):
    A = radon.siddon_matrix(48, 60, 2, 69)
    T = spmv.ThreadedCSR(A, threads)
    x = inputs.random_vector(A.shape[1], 21)
    y = inputs.random_vector(A.shape[0], 22)
    np.testing.assert_array_equal(T @ x, A @ x)
    np.testing.assert_array_equal(T.T @ y, A.T @ y)
    assert T.T.T is T


def test_threaded_products_fall_back_for_complex_and_matrices():
    A = radon.siddon_matrix(16, 12, 1, 23)
    T = spmv.ThreadedCSR(A, 4)
    z = inputs.random_vector(A.shape[1], 23) + 1j * inputs.random_vector(A.shape[1], 24)
    np.testing.assert_allclose(T @ z, A @ z, rtol=1e-15, atol=1e-15)
    np.testing.assert_array_equal((T @ z).real, A @ z.real)
    X = inputs.random_vector(A.shape[1] * 3, 25).reshape(A.shape[1], 3)
    np.testing.assert_array_equal(T @ X, A @ X)
    with pytest.raises(ValueError):
        T @ np.zeros(A.shape[1] + 1)


def test_split_bregman_with_threaded_products_is_unchanged():
    n = 32
    A = radon.siddon_matrix(n, 45, 1, 46)
    f = A @ inputs.ellipse_phantom(n, 5).ravel()
    plain = tv.split_bregman(A, f, (n, n), 1.0, 0.5, 3, 6)
    threaded = tv.split_bregman(spmv.ThreadedCSR(A, 5), f, (n, n), 1.0, 0.5, 3, 6)
    np.testing.assert_array_equal(threaded["u"], plain["u"])
