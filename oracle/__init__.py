"""FP64 CPU oracle for the R-ChFSI filter path (TEST INFRASTRUCTURE ONLY).

Plain, slow, obviously correct NumPy/SciPy code written from the paper
(arXiv 2605.30128, "Towards Exascale Fully Relativistic Pseudopotential DFT
... Residual-Based Subspace Iteration").  It assembles the finite-element
Hamiltonian H and the lumped mass M as explicit (sparse) matrices and runs
the ChFSI and R-ChFSI recurrences, Cholesky-QR, Rayleigh-Ritz and the
eigensolver loop step by step in the paper's order and notation.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it, and it
shares no code with the GPU library: only the seeded input generators in
``workloads`` serve both.

Parity status of each function is stated in its docstring; every function is
pinned by at least one CPU test in ``tests/test_oracle_*.py`` against a closed
form, an invariant, a library routine or brute force.
"""
from .gll import gll_nodes_weights, lagrange_derivative_matrix
from .mesh import Mesh
from .hamiltonian import Hamiltonian, soc_delta, p_orbital_L
from .chebyshev import filter_scalars, ritz_filter_values, chebyshev_filter_closed_form
from .filters import chfsi_filter, rchfsi_filter, residual
from .lanczos import lanczos_bounds
from .rr import cholqr, cholqr2, rayleigh_ritz
from .eigensolver import rchfsi_eigensolver
from .adjoint import rchfsi_filter_adjoint, ritz_loss_head
from .fullmass import FullMassHamiltonian, lagrange_tables
from .poisson import laplacian, poisson_rhs, chebyshev_jacobi, pcg
from .bfp import bfp_encode, bfp_decode, bfp_encode_block, bfp_decode_block, bfp_layout, bfp_stream_bytes

__all__ = [
    "gll_nodes_weights", "lagrange_derivative_matrix", "Mesh", "Hamiltonian", "soc_delta",
    "p_orbital_L", "filter_scalars", "ritz_filter_values", "chebyshev_filter_closed_form",
    "chfsi_filter", "rchfsi_filter", "residual", "lanczos_bounds", "cholqr", "cholqr2",
    "rayleigh_ritz", "rchfsi_eigensolver", "rchfsi_filter_adjoint", "ritz_loss_head",
    "FullMassHamiltonian", "lagrange_tables", "laplacian", "poisson_rhs", "chebyshev_jacobi", "pcg",
    "bfp_encode", "bfp_decode", "bfp_encode_block", "bfp_decode_block", "bfp_layout", "bfp_stream_bytes",
]
