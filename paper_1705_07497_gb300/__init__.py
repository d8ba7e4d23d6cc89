"""GB300-native sparse-operator CT reconstruction (Barnard & Archibald, arXiv 1705.07497).

The compute path lives in ``libct.so`` (CUDA, sm_103a) behind the C ABI of
``include/ct.h``; ``ct`` is the thin ctypes binding to it, ``autograd`` wraps
the forward/adjoint pair as differentiable torch operations, and ``inputs``
makes seeded synthetic phantoms and noise.  Importing the package does not
load the shared library; the first call into ``ct`` does, and it raises if
the library has not been built.
"""

__all__ = ["ct", "inputs"]
