"""GB300 (sm_103a) implementation of Z2-graded fermionic tensor network
contraction (arXiv:2410.02215): the block-sparse fermionic tensordot, the
sector-wise QR/SVD bond compression and the contraction-tree executor, all
behind the C ABI of libftn (include/ftn.h).  ``ftn`` is the ctypes binding."""
from . import ftn  # noqa: F401

__all__ = ["ftn"]
