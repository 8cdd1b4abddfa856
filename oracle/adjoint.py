"""Reverse-mode derivative of the R-ChFSI filter and of a Ritz-value loss.

The paper has no adjoint; this is the transpose of the forward recurrence
(Eq. rChFSIrecurrence with Z_0 = 0, Z_1 = sigma_1 R / e, R = H X - M X Lambda,
Y_q = D^{-1} Z_q + X Lambda_q) with X, Lambda and the filter bounds held
constant.  Parameters are the quadrature-point fields V, B (Eq. hloc) and the
spin-orbit couplings h (Eq. hnloc).

Forward quantities are stored in full (no checkpointing), so this is an
independent check of the checkpointed GPU adjoint.  With dL = Re tr(Ybar^H dY):
  Zbar_q = D^{-1} Ybar
  for k = q-1 .. 1 (a_k = 2 sigma_{k+1}/e, b_k = sigma_k sigma_{k+1}):
      dH   <- a_k  Zbar_{k+1} (D^{-1} Z_k)^H
      Zbar_k     += a_k (D^{-1} H - c) Zbar_{k+1}
      Zbar_{k-1} -= b_k Zbar_{k+1}
      Rbar       += a_k Zbar_{k+1} Lambda_k
  Rbar += (sigma_1 / e) Zbar_1;   dH <- Rbar X^H

Parity: pinned by central finite differences and a directional
(dot-product) test on small meshes (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .chebyshev import filter_scalars, ritz_filter_values
from .filters import rchfsi_filter


def rchfsi_filter_adjoint(Hop, X, lam, lmin, lT, lmax, q, Ybar):
    """Node-level gradients (gV, gB, gh) of Re tr(Ybar^H Y_q) and the forward Y_q."""
    c, e, sigma = filter_scalars(lmin, lT, lmax, q)
    Y, Z, R = rchfsi_filter(Hop, X, lam, lmin, lT, lmax, q, return_history=True)
    Lk = ritz_filter_values(lam, lmin, lT, lmax, q)
    Dinv = 1.0 / Hop.Mdiag[:, None]
    gV = np.zeros(Hop.nnodes)
    gB = np.zeros((3, Hop.nnodes))
    gh = np.zeros((len(Hop.projectors), 2))

    def acc(W, U, wgt):
        nonlocal gV, gB, gh
        a, b, cc = Hop.bilinear_grads(W, U, wgt)
        gV += a
        gB += b
        gh += cc

    Zbar = [np.zeros_like(X) for _ in range(q + 1)]
    Zbar[q] = Dinv * Ybar
    Rbar = np.zeros_like(X)
    for k in range(q - 1, 0, -1):
        a = 2.0 * sigma[k + 1] / e
        b = sigma[k] * sigma[k + 1]
        acc(Zbar[k + 1], Dinv * Z[k], a)
        Zbar[k] += a * (Dinv * Hop.apply(Zbar[k + 1]) - c * Zbar[k + 1])
        Zbar[k - 1] -= b * Zbar[k + 1]
        Rbar += a * Zbar[k + 1] * Lk[k][None, :]
    Rbar += (sigma[1] / e) * Zbar[1]
    acc(Rbar, X, 1.0)
    return (gV, gB, gh), Y


def ritz_loss_head(Hop, Y, G, nlow):
    """L = sum_{j < nlow} theta_j + Re <G, Y>_F with theta the Ritz values of span(Y).

    Returns (L, Ybar, direct) where Ybar = dL/dY (as Re tr(Ybar^H dY)) and
    direct = node-level gradients of sum_j x_j^H dH x_j (the explicit H
    dependence of the Ritz values).
    """
    A = Y.conj().T @ Hop.apply(Y)
    S = Y.conj().T @ (Hop.Mdiag[:, None] * Y)
    A = 0.5 * (A + A.conj().T)
    S = 0.5 * (S + S.conj().T)
    theta, Q = sla.eigh(A, S)                       # Q^H S Q = I
    Xr = Y @ Q[:, :nlow]
    L = float(np.sum(theta[:nlow]) + np.real(np.vdot(G, Y)))
    HX = Hop.apply(Xr)
    MX = Hop.Mdiag[:, None] * Xr
    Ybar = 2.0 * (HX - MX * theta[None, :nlow]) @ Q[:, :nlow].conj().T + G
    direct = Hop.bilinear_grads(Xr, Xr, 1.0)
    return L, Ybar, direct
