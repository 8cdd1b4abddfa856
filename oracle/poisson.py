"""Periodic FE Poisson solve by preconditioned CG with a Chebyshev-Jacobi preconditioner
(Section III-B-1; Algorithm pcg_fusion) (TEST INFRASTRUCTURE ONLY).

K is the FE discrete Laplacian K_IJ = int grad N_I . grad N_J on the periodic GLL mesh (twice
the kinetic matrix of Eq. hloc); the right-hand side of -lap V = 4 pi rho is
f_I = 4 pi int N_I rho, here by the GLL rule, f_I = 4 pi M_I rho(x_I).  The periodic K is
singular (constant null space), so f is taken with zero sum and the solution with zero
mean.

PCG in the paper's arrangement: r = K x - f; each iteration w = K p, eta = p.w,
alpha = delta / eta, x += alpha p and r += alpha w (one fused pass), z = P^-1 r,
(delta_new, gamma) = (r.z, r.r) (one fused reduction), beta = delta_new / delta,
p = -z + beta p, stop when sqrt(gamma) < eps.

Preconditioner: P^-1 = chi(A) K_diag^-1 with A = K_diag^-1 K and K_diag = diag(K), chi the
degree-m polynomial of Chebyshev semi-iteration for A y = g from y = 0 on the interval
[a, b] (the textbook three-term recurrence): 1 - lambda chi(lambda) =
T_m((theta - lambda)/delta) / T_m(theta/delta), theta = (a + b)/2, delta = (b - a)/2, the
minimax residual polynomial on [a, b].  The interval is an input: the paper estimates the
top of the spectrum of A by a short Lanczos run; the bottom is a chosen fraction of it.

Parity: pinned in tests/test_oracle_poisson.py: the preconditioner against the closed form
of the residual polynomial on exact eigenvectors of A; the PCG iterates against scipy's
CG with the same preconditioner; the discrete solution against a dense solve; the plane-wave
charge against the continuum solution, converging in p; fewer iterations than Jacobi PCG.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Mesh


def laplacian(mesh: Mesh) -> sp.csr_matrix:
    """K_IJ = int grad N_I . grad N_J (scalar, nnodes x nnodes)."""
    return (2.0 * mesh.kinetic()).tocsr()


def poisson_rhs(mesh: Mesh, rho_nodes: np.ndarray) -> np.ndarray:
    """f_I = 4 pi M_I rho(x_I) (GLL rule), shifted to zero sum (the solvability condition)."""
    f = 4.0 * np.pi * mesh.lumped_mass() * np.asarray(rho_nodes, dtype=np.float64)
    return f - f.mean()


def chebyshev_jacobi(K, Kdiag: np.ndarray, r: np.ndarray, m: int, a: float, b: float) -> np.ndarray:
    """z = chi(A) Kdiag^-1 r: m steps of Chebyshev semi-iteration for A y = Kdiag^-1 r, y_0 = 0."""
    if not (0.0 < a < b):
        raise ValueError("need 0 < a < b")
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma1 = theta / delta
    g = r / Kdiag
    y = np.zeros_like(g)
    res = g.copy()                        # g - A y
    rho = 1.0 / sigma1
    d = res / theta
    for _ in range(m):
        y = y + d
        res = res - (K @ d) / Kdiag
        rho_next = 1.0 / (2.0 * sigma1 - rho)
        d = rho_next * rho * d + (2.0 * rho_next / delta) * res
        rho = rho_next
    return y


def pcg(K, f: np.ndarray, precond, eps: float, maxit: int, x0: np.ndarray | None = None):
    """PCG in the order of Algorithm pcg_fusion; returns (x, iterations, history of ||r||)."""
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    r = K @ x - f
    z = precond(r)
    delta = float(r @ z)
    p = -z
    hist = [float(np.sqrt(r @ r))]
    it = 0
    while hist[-1] >= eps and it < maxit:
        w = K @ p
        eta = float(p @ w)
        alpha = delta / eta
        x = x + alpha * p
        r = r + alpha * w
        z = precond(r)
        delta_new, gamma = float(r @ z), float(r @ r)
        beta = delta_new / delta
        delta = delta_new
        p = -z + beta * p
        it += 1
        hist.append(float(np.sqrt(gamma)))
    return x, it, hist
