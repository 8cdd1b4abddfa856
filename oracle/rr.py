"""Cholesky-QR orthonormalisation and the Rayleigh-Ritz step (Algorithm 1, RR step; Section III-C-4).

The paper solves the projected generalized problem
(Y^H H Y) Q = (Y^H M Y) Q Lambda and rotates X = Y Q.  Here Y is first made
M-orthonormal by Cholesky-QR applied twice (S = Y^H M Y = L L^H,
Y <- Y L^{-H}), after which the projected problem is the standard Hermitian
eigenproblem of A = Y^H H Y; both routes give the same Ritz pairs.

Parity: pinned against scipy.linalg.eigh(A, S) on the unorthonormalised
block and against dense brute force (tests/test_oracle_filters.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def cholqr(Y: np.ndarray, Mdiag: np.ndarray) -> np.ndarray:
    S = Y.conj().T @ (Mdiag[:, None] * Y)
    S = 0.5 * (S + S.conj().T)
    L = np.linalg.cholesky(S)                       # S = L L^H, L lower
    # Y L^{-H}:  solve L Z^H = Y^H  ->  Z = Y L^{-H}
    return sla.solve_triangular(L, Y.conj().T, lower=True).conj().T


def cholqr2(Y: np.ndarray, Mdiag: np.ndarray) -> np.ndarray:
    return cholqr(cholqr(Y, Mdiag), Mdiag)


def cholqr_full(Y: np.ndarray, mass_apply) -> np.ndarray:
    """Cholesky-QR with a full mass: S = Y^H (M Y) = L L^H, Y <- Y L^{-H}."""
    S = Y.conj().T @ mass_apply(Y)
    S = 0.5 * (S + S.conj().T)
    L = np.linalg.cholesky(S)
    return sla.solve_triangular(L, Y.conj().T, lower=True).conj().T


def rayleigh_ritz(Hop, Y: np.ndarray):
    """Return (X, theta): Y is M-orthonormalised by CholQR2 (the full M where the operator
    has one), then A = Y^H H Y is diagonalised."""
    if hasattr(Hop, "mass_apply"):
        Yo = cholqr_full(cholqr_full(Y, Hop.mass_apply), Hop.mass_apply)
    else:
        Yo = cholqr2(Y, Hop.Mdiag)
    A = Yo.conj().T @ Hop.apply(Yo)
    A = 0.5 * (A + A.conj().T)
    theta, Q = np.linalg.eigh(A)
    return Yo @ Q, theta
