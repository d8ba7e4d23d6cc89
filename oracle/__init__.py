"""FP64 CPU oracle for sparse-operator CT reconstruction (Barnard & Archibald).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it; the library itself never does, and the two
share no code (no kernels, headers, helpers or tables).

Contents
  radon      exact Siddon system matrix A = M R (Sec. 1, Eq. objmin) in FP64,
             built by ``siddon.c``; a per-pixel clipping brute force for tiny
             images; FP16 row-scale quantisation of A.
  tv         forward-difference gradient and its adjoint, conjugate gradients,
             anisotropic-TV split Bregman (Sec. 2, Eq. SB_solve; Sec. 4), the
             Chambolle-Pock resolvent (Sec. 2, Eq. PD_resolve), and the sparse
             surrogate T (Sec. 3.2, Eq. def_sparse_surr / surr_SBupd).
  spmv       the CSR products on several host threads (rows summed in
             storage order, so the result does not depend on the threads).
  fourier    the Fourier-domain data term (Sec. 2, Eq. four_obj): the exact
             nonuniform DFT on polar samples, the data's 1-D DFTs, Gaussian
             gridding and the fused matrix B* B (Sec. 3.1, Eq. fusedop).

Every floating-point result is FP64.  Readings of the paper where it is
silent or garbled are stated in the docstring of the function that takes them.
"""

from . import fourier, radon, spmv, tv  # noqa: F401
