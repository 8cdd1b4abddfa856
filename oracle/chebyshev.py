"""Scalar parts of the Chebyshev filter (Section III-B-2, Eq. ChFSIrecurrence and the text after it).

c = (lambda_max + lambda_T)/2, e = (lambda_max - lambda_T)/2,
sigma_1 = e / (lambda_min - c), sigma_{k+1} = 1 / (2/sigma_1 - sigma_k),
C_k(x) = T_k((x - c)/e) / T_k((lambda_min - c)/e).
Lambda_k = C_k(Lambda) is propagated with the same three-term recurrence
(text after Eq. rChFSIrecurrence): Lambda_0 = 1, Lambda_1 = sigma_1 (Lambda - c)/e,
Lambda_{k+1} = (2 sigma_{k+1}/e)(Lambda - c) Lambda_k - sigma_k sigma_{k+1} Lambda_{k-1}.

Parity: the recurrence is pinned against the closed form C_k evaluated with
numpy's Chebyshev-series routine (tests/test_oracle_filters.py).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import chebyshev as npcheb


def filter_scalars(lmin: float, lT: float, lmax: float, q: int):
    """Return (c, e, sigma) with sigma[k] = sigma_k for k = 1..q (sigma[0] unused)."""
    if not (lmin < lT < lmax):
        raise ValueError("need lambda_min < lambda_T < lambda_max")
    c = 0.5 * (lmax + lT)
    e = 0.5 * (lmax - lT)
    sigma = np.zeros(q + 1)
    sigma[1] = e / (lmin - c)
    for k in range(1, q):
        sigma[k + 1] = 1.0 / (2.0 / sigma[1] - sigma[k])
    return c, e, sigma


def ritz_filter_values(lam: np.ndarray, lmin: float, lT: float, lmax: float, q: int) -> np.ndarray:
    """Lambda_k = C_k(Lambda) for k = 0..q by the three-term recurrence; shape (q + 1, len(lam))."""
    lam = np.asarray(lam, dtype=np.float64)
    c, e, sigma = filter_scalars(lmin, lT, lmax, q)
    out = np.zeros((q + 1, lam.size))
    out[0] = 1.0
    if q >= 1:
        out[1] = sigma[1] * (lam - c) / e
    for k in range(1, q):
        out[k + 1] = (2.0 * sigma[k + 1] / e) * (lam - c) * out[k] - sigma[k] * sigma[k + 1] * out[k - 1]
    return out


def chebyshev_filter_closed_form(lam, lmin: float, lT: float, lmax: float, k: int) -> np.ndarray:
    """C_k(lambda) = T_k((lambda - c)/e) / T_k((lambda_min - c)/e) via numpy.polynomial.chebyshev."""
    c = 0.5 * (lmax + lT)
    e = 0.5 * (lmax - lT)
    coef = np.zeros(k + 1)
    coef[k] = 1.0
    return npcheb.chebval((np.asarray(lam, float) - c) / e, coef) / npcheb.chebval((lmin - c) / e, coef)
