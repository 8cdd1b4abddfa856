"""Spectral upper bound for the filter from a short Lanczos run.

The filter needs lambda_max, an upper bound on the spectrum of M^{-1} H
(Section III-B-2); the paper selects the interval from an estimate of the
largest eigenvalue (Section IV-F) and uses a short Lanczos run for the
spectral bounds of its preconditioner (Section III-C-1).  Reading used here:
m steps of plain Lanczos (no re-orthogonalisation) on the Hermitian
D^{-1/2} H D^{-1/2}, which has the spectrum of D^{-1} H, from a given start
vector; lambda_max = max Ritz value + |beta_m|.

Parity: pinned by brute force (dense eigvalsh) on small meshes: the bound is
above the largest eigenvalue and, after as many steps as the dimension, the
Ritz values are the eigenvalues (tests/test_oracle_filters.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def lanczos_bounds(Hop, v0: np.ndarray, m: int):
    """Return (theta_min, theta_max + |beta_m|, alphas, betas)."""
    s = 1.0 / np.sqrt(Hop.Mdiag)

    def op(v):
        return s * Hop.apply(s * v)

    v = np.asarray(v0, dtype=np.complex128).copy()
    v /= np.linalg.norm(v)
    vprev = np.zeros_like(v)
    beta_prev = 0.0
    alphas, betas = [], []
    for _ in range(m):
        w = op(v) - beta_prev * vprev
        alpha = float(np.real(np.vdot(v, w)))
        w = w - alpha * v
        beta = float(np.linalg.norm(w))
        alphas.append(alpha)
        betas.append(beta)
        vprev, v, beta_prev = v, w / beta, beta
    theta = sla.eigh_tridiagonal(np.array(alphas), np.array(betas[:-1]), eigvals_only=True)
    return float(theta.min()), float(theta.max() + abs(betas[-1])), np.array(alphas), np.array(betas)
