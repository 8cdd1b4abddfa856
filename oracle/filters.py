"""ChFSI and R-ChFSI filters, written step by step (Section III-B-2).

chfsi_filter: Eq. ChFSIrecurrence with Y_0 = X and
Y_1 = sigma_1 (M^{-1} H - c I) X / e; here M is the GLL-lumped diagonal so
M^{-1} is applied exactly.

rchfsi_filter: Eq. rChFSIrecurrence with Z_0 = 0, Z_1 = sigma_1 R / e,
R = H X - M X Lambda computed in FP64 (with the full mass where the operator
has one), Lambda_k propagated in FP64 by the same recurrence, and the recovery
Y_q = D^{-1} Z_q + X Lambda_q (Algorithm 1, the recover step).  D defaults to
the operator's diagonal (M itself on the lumped mesh).

Parity: R-ChFSI equals ChFSI exactly when D = M (a closed-form identity of the
two recurrences); both reproduce Y_q = X C_q(Lambda) on exact eigenvectors
(tests/test_oracle_filters.py).
"""
from __future__ import annotations

import numpy as np

from .chebyshev import filter_scalars, ritz_filter_values


def mass_times(Hop, X: np.ndarray) -> np.ndarray:
    """M X: the full mass where the operator has one (``mass_apply``), else the diagonal M."""
    if hasattr(Hop, "mass_apply"):
        return Hop.mass_apply(X)
    return Hop.Mdiag[:, None] * X if X.ndim == 2 else Hop.Mdiag * X


def residual(Hop, X: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """R = H X - M X Lambda (Algorithm 1, residual step)."""
    return Hop.apply(X) - mass_times(Hop, X) * np.asarray(lam)[None, :]


def chfsi_filter(Hop, X: np.ndarray, lmin: float, lT: float, lmax: float, q: int,
                 exact_mass: bool = False) -> np.ndarray:
    """Y_q = C_q(M^{-1} H) X by Eq. ChFSIrecurrence (FP64).

    M^{-1} is applied as the inverse of the operator's diagonal (``Mdiag``: M itself
    on the lumped mesh, the diagonal D in place of a full M); with exact_mass the
    full mass is solved exactly (``mass_solve``)."""
    c, e, sigma = filter_scalars(lmin, lT, lmax, q)
    Minv = 1.0 / Hop.Mdiag[:, None]

    def op(Y):  # (M^{-1} H - c) Y
        if exact_mass:
            return Hop.mass_solve(Hop.apply(Y)) - c * Y
        return Minv * Hop.apply(Y) - c * Y

    Yprev = X.copy()
    Y = (sigma[1] / e) * op(X)
    for k in range(1, q):
        Ynext = (2.0 * sigma[k + 1] / e) * op(Y) - sigma[k] * sigma[k + 1] * Yprev
        Yprev, Y = Y, Ynext
    return Y


def rchfsi_filter(Hop, X: np.ndarray, lam: np.ndarray, lmin: float, lT: float, lmax: float, q: int,
                  Ddiag: np.ndarray | None = None, return_history: bool = False):
    """Y_q by Eq. rChFSIrecurrence and the recovery step (FP64).

    With return_history the list [Z_0, ..., Z_q] and R are returned as well.
    """
    c, e, sigma = filter_scalars(lmin, lT, lmax, q)
    lam = np.asarray(lam, dtype=np.float64)
    D = Hop.Mdiag if Ddiag is None else np.asarray(Ddiag, float)
    Dinv = 1.0 / D[:, None]
    R = residual(Hop, X, lam)
    Lk = ritz_filter_values(lam, lmin, lT, lmax, q)       # Lambda_k, k = 0..q
    Z = [np.zeros_like(X), (sigma[1] / e) * R]
    for k in range(1, q):
        a = 2.0 * sigma[k + 1] / e
        Znext = (a * Hop.apply(Dinv * Z[k]) - a * c * Z[k] - sigma[k] * sigma[k + 1] * Z[k - 1]
                 + a * R * Lk[k][None, :])
        Z.append(Znext)
    Y = Dinv * Z[q] + X * Lk[q][None, :]
    if return_history:
        return Y, Z, R
    return Y
