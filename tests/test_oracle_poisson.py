"""Pins of the Poisson PCG oracle (Section III-B-1; Algorithm pcg_fusion).

Independent references: the closed form of the Chebyshev residual polynomial (numpy's
Chebyshev series) on exact eigenvectors, scipy's conjugate-gradient iterates with the same
preconditioner, a dense solve, and the continuum solution of a plane-wave charge.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as C

from oracle import Mesh
from oracle.poisson import chebyshev_jacobi, laplacian, pcg, poisson_rhs


def _problem(n=2, L=6.0, p=3, seed=0):
    mesh = Mesh(n, L, p)
    K = laplacian(mesh)
    rng = np.random.default_rng(seed)
    f = poisson_rhs(mesh, rng.standard_normal(mesh.nnodes))
    return mesh, K, K.diagonal().copy(), f


def test_laplacian_is_the_kinetic_matrix_doubled_and_annihilates_constants():
    mesh, K, Kd, _ = _problem()
    np.testing.assert_allclose(K @ np.ones(mesh.nnodes), 0.0, atol=1e-12)
    Kdense = K.toarray()
    np.testing.assert_allclose(Kdense, Kdense.T, atol=1e-14)
    ev = np.linalg.eigvalsh(Kdense)
    assert abs(ev[0]) < 1e-11 and ev[1] > 1e-3            # one zero mode, the rest positive


@pytest.mark.parametrize("m", [1, 3, 6])
def test_chebyshev_preconditioner_matches_its_residual_polynomial(m):
    mesh, K, Kd, _ = _problem(p=2)
    lam, V = sla.eigh(K.toarray(), np.diag(Kd))             # K v = lambda Kdiag v
    b = 1.05 * lam[-1]
    a = b / 15.0
    theta, delta = 0.5 * (a + b), 0.5 * (b - a)
    Tm = np.zeros(m + 1)
    Tm[m] = 1.0
    for j in range(1, lam.size, 7):                         # a spread of eigenvectors, lambda > 0
        l = lam[j]
        chi = (1.0 - C.chebval((theta - l) / delta, Tm) / C.chebval(theta / delta, Tm)) / l
        z = chebyshev_jacobi(K, Kd, Kd * V[:, j], m, a, b)
        np.testing.assert_allclose(z, chi * V[:, j], atol=1e-10 * np.abs(V[:, j]).max())


def test_pcg_iterates_match_scipy_cg():
    mesh, K, Kd, f = _problem(p=3)
    b = 1.05 * spla.eigsh(spla.LinearOperator(K.shape, matvec=lambda v: (K @ v) / Kd), k=1,
                          which="LM", return_eigenvectors=False)[0]
    pre = lambda r: chebyshev_jacobi(K, Kd, r, 4, b / 20.0, b)
    ours = []
    for k in range(1, 7):
        x, it, _ = pcg(K, f, pre, 0.0, k)
        assert it == k
        ours.append(x)
    ref = []
    spla.cg(K, f, x0=np.zeros_like(f), rtol=0.0, atol=0.0, maxiter=6,
            M=spla.LinearOperator(K.shape, matvec=pre), callback=lambda xk: ref.append(xk.copy()))
    for x, y in zip(ours, ref):
        np.testing.assert_allclose(x, y, atol=1e-9 * np.abs(y).max())


def test_pcg_solution_matches_a_dense_solve_and_beats_jacobi():
    mesh, K, Kd, f = _problem(n=3, p=3)
    b = 1.05 * spla.eigsh(spla.LinearOperator(K.shape, matvec=lambda v: (K @ v) / Kd), k=1,
                          which="LM", return_eigenvectors=False)[0]
    x, it_cheb, hist = pcg(K, f, lambda r: chebyshev_jacobi(K, Kd, r, 5, b / 20.0, b), 1e-10, 500)
    assert hist[-1] < 1e-10
    xd = np.linalg.lstsq(K.toarray(), f, rcond=None)[0]      # minimum-norm (zero-mean) solution
    np.testing.assert_allclose(x - x.mean(), xd - xd.mean(), atol=1e-8 * np.abs(xd).max())
    _, it_jac, _ = pcg(K, f, lambda r: r / Kd, 1e-10, 2000)
    assert it_cheb < it_jac / 2


def test_plane_wave_charge_converges_to_the_continuum_solution():
    # -lap V = 4 pi cos(2 pi x / L)  ->  V = 4 pi (L / 2 pi)^2 cos(2 pi x / L)
    L = 6.0
    errs = []
    for p in (2, 3, 4, 5):
        mesh = Mesh(2, L, p)
        K = laplacian(mesh)
        Kd = K.diagonal().copy()
        x = mesh.node_coords()[:, 0]
        f = poisson_rhs(mesh, np.cos(2 * np.pi * x / L))
        b = 1.05 * spla.eigsh(spla.LinearOperator(K.shape, matvec=lambda v: (K @ v) / Kd), k=1,
                              which="LM", return_eigenvectors=False)[0]
        V, _, hist = pcg(K, f, lambda r: chebyshev_jacobi(K, Kd, r, 5, b / 20.0, b), 1e-11, 500)
        M = mesh.lumped_mass()
        V = V - (M @ V) / M.sum()
        exact = 4 * np.pi * (L / (2 * np.pi)) ** 2 * np.cos(2 * np.pi * x / L)
        errs.append(np.abs(V - exact).max() / np.abs(exact).max())
    assert all(errs[i] > 3 * errs[i + 1] for i in range(3)) and errs[-1] < 1e-3
