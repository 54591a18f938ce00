"""CPU oracle for the K-GRAPE hot path (complex128, NumPy).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import it.  The CUDA library and its Python
binding never import, call or link anything here, and this package imports nothing
from them; the two share only the seeded input generators, which hold none of the
method's arithmetic.

Modules (each function cites the passage of the paper it follows):

* ``chain``  - matrix-free open XXZ chain H0 + u Hc (Sec. 3.1, Eq. H01, Eq. htot)
* ``krylov`` - Lanczos basis with full re-orthogonalisation and the Krylov time
               step exp(-i sigma dt T) e_1 via eigh (Appendix A)
* ``grape``  - forward sweep, overlap, backward co-state sweep, per-slice overlaps
               and the zeroth-order / centred gradients (Sec. 2, App. B)
* ``dense``  - dense eigendecomposition propagators and the exact gradient for
               small chains (App. B)
* ``sector`` - the chain in a parity-excitation subspace (Sec. 3.1): sector states,
               parity eigenbasis Q, H_red = Q H Q^T, with the ``Chain`` interface

Every function is pinned by tests marked "not gpu" against results that do not
come from the oracle itself (Kronecker-product Hamiltonians, closed forms at L=1
and L=2, scipy's expm, invariants, finite differences, error orders).
"""
from .chain import Chain
from .krylov import expm_e1, krylov_step, lanczos, tridiag
from .grape import evaluate, forward, overlaps_G, segment_forward_backward
from .dense import exact_fidelity, exact_forward, exact_gradient
from .sector import SectorChain, paper_chain

__all__ = [
    "Chain", "expm_e1", "krylov_step", "lanczos", "tridiag", "evaluate", "forward",
    "overlaps_G", "segment_forward_backward", "exact_fidelity", "exact_forward", "exact_gradient",
    "SectorChain", "paper_chain",
]
