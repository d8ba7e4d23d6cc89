"""Threaded FP64 CSR products for the oracle's large runs.

Test infrastructure only (see the package docstring).

``ThreadedCSR(A)`` wraps a scipy CSR matrix so that ``A @ x`` and
``A.T @ y`` of real FP64 vectors run the plain row loop of ``spmv.c`` on
several host threads; every row is still summed in storage order by one
thread, so the products equal a sequential loop's whatever the thread count.
A complex vector (complex-step derivatives) takes two real products, one per
part; anything else (2-D operands) falls back to scipy.  The solvers in
``tv`` take any object with ``@`` and ``.T``, so a wrapped matrix drops in
for the plain one.
"""

import os

import numpy as np
import scipy.sparse as sp

from . import _native


def default_threads():
    return max(1, int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1)))


class ThreadedCSR:
    def __init__(self, A, threads=None, _transpose=None):
        A = sp.csr_matrix(A)
        A.sort_indices()
        self.A = A
        self.shape = A.shape
        self.threads = default_threads() if threads is None else int(threads)
        self._indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self._indices = np.ascontiguousarray(A.indices, dtype=np.int32)
        self._data = np.ascontiguousarray(A.data, dtype=np.float64)
        self._T = _transpose

    @property
    def T(self):
        if self._T is None:
            self._T = ThreadedCSR(self.A.T.tocsr(), self.threads, _transpose=self)
        return self._T

    def __matmul__(self, x):
        x = np.asarray(x)
        if x.ndim == 1 and x.dtype == np.complex128:
            # A is real: the real and imaginary parts are two real products,
            # each row summed in the same order as the complex product
            return self @ np.ascontiguousarray(x.real) + 1j * (self @ np.ascontiguousarray(x.imag))
        if x.ndim != 1 or x.dtype != np.float64:
            return self.A @ x
        x = np.ascontiguousarray(x)
        if x.shape[0] != self.shape[1]:
            raise ValueError("dimension mismatch")
        y = np.empty(self.shape[0])
        _native.spmv_lib().oracle_csr_matvec(self.shape[0], self._indptr.ctypes.data, self._indices.ctypes.data,
                                             self._data.ctypes.data, x.ctypes.data, y.ctypes.data, self.threads)
        return y
