"""Algorithm 1: the R-ChFSI eigensolver for H X = M X Lambda.

Steps in the paper's order: while max_j ||H x_j - eps_j M x_j|| >= tau:
residual (FP64); filter (Eq. rChFSIrecurrence); recover Y_q; Rayleigh-Ritz
(projected eigenproblem, subspace rotation); update lambda_min and lambda_T
from the new Ritz values.  Readings where the paper is silent: the initial Ritz
pairs come from a Rayleigh-Ritz step on the start block, and after each cycle
lambda_min = min Lambda, lambda_T = max Lambda; lambda_max is fixed; the
block carries a buffer of extra vectors above the wanted ones, and the
stopping test covers the wanted ones.

Parity: converged Ritz values are pinned against dense brute force on small
meshes (tests/test_oracle_filters.py).
"""
from __future__ import annotations

import numpy as np

from .filters import chfsi_filter, rchfsi_filter, residual
from .rr import rayleigh_ritz


def residual_norms(Hop, X, lam):
    return np.linalg.norm(residual(Hop, X, lam), axis=0)


def rchfsi_eigensolver(Hop, X0: np.ndarray, q: int, lmax: float, tol: float, max_cycles: int,
                       mode: str = "rchfsi", lmin: float | None = None, nwanted: int | None = None):
    """Run Algorithm 1; returns (X, Lambda, history) with one dict per cycle.

    The stopping test runs over the lowest ``nwanted`` Ritz pairs (default:
    all); the remaining vectors of the block are a convergence buffer.
    """
    nw = X0.shape[1] if nwanted is None else int(nwanted)
    X, lam = rayleigh_ritz(Hop, X0)
    lo = float(lam.min()) if lmin is None else lmin
    lT = float(lam.max())
    history = []
    for cycle in range(max_cycles):
        res = residual_norms(Hop, X, lam)
        history.append(dict(cycle=cycle, ritz=lam.copy(), maxres=float(res[:nw].max()), lmin=lo, lT=lT))
        if res[:nw].max() < tol:
            break
        if mode == "rchfsi":
            Y = rchfsi_filter(Hop, X, lam, lo, lT, lmax, q)
        elif mode == "chfsi_exact_mass":
            Y = chfsi_filter(Hop, X, lo, lT, lmax, q, exact_mass=True)
        else:
            Y = chfsi_filter(Hop, X, lo, lT, lmax, q)
        X, lam = rayleigh_ritz(Hop, Y)
        lo = float(lam.min()) if lmin is None else lmin
        lT = float(lam.max())
    else:
        res = residual_norms(Hop, X, lam)
        history.append(dict(cycle=max_cycles, ritz=lam.copy(), maxres=float(res[:nw].max()), lmin=lo, lT=lT))
    return X, lam, history
