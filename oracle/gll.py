"""Gauss-Lobatto-Legendre nodes, weights and the Lagrange derivative matrix.

The paper's basis (Section III-A, Eq. FEWfns) is the tensor product of 1D
Lagrange polynomials of degree p on GLL nodes.  Pinned in
tests/test_oracle_fem.py against the textbook closed forms for p = 2, 3, 4
(tests/golden/gll_closed_forms.txt), quadrature exactness up to degree 2p-1,
and exact differentiation of polynomials of degree <= p.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def gll_nodes_weights(p: int):
    """GLL nodes xi_0 = -1 < ... < xi_p = 1 and weights on [-1, 1].

    Interior nodes are the roots of P_p'(x); the weights are
    w_a = 2 / (p (p + 1) P_p(xi_a)^2).
    """
    if p < 1:
        raise ValueError("degree p must be >= 1")
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    interior = np.sort(np.real(npleg.legroots(npleg.legder(cp)))) if p > 1 else np.zeros(0)
    xi = np.concatenate([[-1.0], interior, [1.0]])
    Pp = npleg.legval(xi, cp)
    w = 2.0 / (p * (p + 1) * Pp * Pp)
    return xi, w


def lagrange_derivative_matrix(xi: np.ndarray) -> np.ndarray:
    """D[q, a] = l_a'(xi_q) for the Lagrange basis l_a on the nodes xi.

    Each l_a is built as the monomial-basis polynomial prod_{m != a}(x - xi_m)
    divided by prod_{m != a}(xi_a - xi_m), then differentiated and evaluated.
    """
    n = len(xi)
    D = np.empty((n, n))
    for a in range(n):
        others = np.delete(xi, a)
        coeffs = nppoly.polyfromroots(others) / np.prod(xi[a] - others)
        D[:, a] = nppoly.polyval(xi, nppoly.polyder(coeffs))
    return D
