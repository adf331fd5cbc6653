"""CPU FP64 oracle for fermionic (Z2-graded) tensor network contraction.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the ``paper_2410_02215_gb300`` package and its CUDA library) never imports,
links or calls anything here, and this package imports nothing from it.

Every graded tensor is embedded densely: a leg with sector dimensions
``(d_even, d_odd)`` has ``d_even + d_odd`` indices, the even ones first, and the
parity of index ``i`` is ``[i >= d_even]``.  Entries outside the
parity-allowed set are zero and stay zero.  The fermionic signs are applied
explicitly to the dense arrays, following the paper (arXiv:2410.02215):

* transposition sign, Eq. (transposition), Sec. II.B;
* contraction by moving contracted legs adjacent, Eq. (standardcontract);
* swap rule and bond parity tensor g, Eqs. (fermiswap)-(swapeq), Fig. 2;
* globally ordered formalism, Eq. (fermionictn), Sec. II.C;
* locally ordered formalism, Eq. (fermionictn2), Sec. II.D;
* index fusion, Sec. IV.A; symmetric QR/SVD truncation, Sec. II.A;
* Fermi-Hubbard Hamiltonian, Eq. (fermi-hubbard-ham), Sec. V;
* the gradient of a contraction with respect to either operand, by its
  definition (one contraction per parity-allowed entry);
* the gradient of the QR/SVD compression, by the reverse-mode rules of its
  steps, and of a closed network's value through its contraction tree and
  compressions (both pinned by finite differences of the forward oracle);
* the cluster approximation of local energy terms, Sec. V (cluster networks
  in the globally ordered formalism, Fig. 4b);
* U(1) x parity tensors (charges whose parity is the charge mod 2, Sec. II.B).

Parity pins: every function is checked by ``tests/test_oracle_*.py`` against
closed forms printed in the paper, textbook reductions (bosonic legs ->
``numpy.einsum``), brute-force sums and exact diagonalisation.  No function
here is "parity unpinned".
"""
from .graded import *  # noqa: F401,F403
from .network import *  # noqa: F401,F403
from .compress import *  # noqa: F401,F403
from .hubbard import *  # noqa: F401,F403
from .adjoint import *  # noqa: F401,F403
from .cluster import *  # noqa: F401,F403
from .compress_adjoint import *  # noqa: F401,F403
from .network_grad import *  # noqa: F401,F403
from .u1 import *  # noqa: F401,F403
