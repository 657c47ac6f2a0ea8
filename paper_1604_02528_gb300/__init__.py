"""GB300 (sm_103a) supernodal selected inversion.

Computes the entries of A^{-1} on the pattern of the LDL^T factor of a sparse
symmetric or complex symmetric matrix by the elimination-tree recursion of
Jacquelin, Lin, Jia, Zhao and Yang (Alg. 1 / Alg. 2), on one GPU, behind the
C ABI of ``include/selinv.h``.  This package is the thin Python side:

* ``_native``  -- ctypes binding, one function per C entry point
* ``api``      -- convenience wrappers (plan from a matrix, torch buffers)
* ``autograd`` -- ``SelInv``: a torch.autograd.Function over factor + selinv

Importing the package does not load the native library; ``_native`` does,
and fails loudly when it is missing.
"""

__all__ = ["build", "native"]


def build(force: bool = False) -> str:
    """Compile libselinv.so in-tree (nvcc, sm_103a)."""
    from . import buildlib as _b
    return _b.build(force=force)


def native():
    """The ctypes binding module (loads libselinv.so)."""
    from . import _native
    return _native
