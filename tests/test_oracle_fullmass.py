"""Pins of the full-consistent-mass oracle (Gauss-Legendre quadrature; Section III-A,
Section III-B-2).

The 1D reference matrices here come from exact polynomial integration (numpy Polynomial
products and antiderivatives), independent of the oracle's quadrature tables; the 3D
operators must reproduce them through the tensor-product structure of the basis, and
the full problem must show the behaviour the paper states: R-ChFSI with a diagonal D in
place of M^-1 reaches the eigenpairs of (H, M), ChFSI with the same D stalls.
"""
import numpy as np
import pytest
import scipy.linalg as sla
from numpy.polynomial import Polynomial as Pn

import workloads
from oracle import Mesh, gll_nodes_weights, lagrange_derivative_matrix
from oracle.eigensolver import rchfsi_eigensolver
from oracle.fullmass import FullMassHamiltonian, lagrange_tables


def lagrange_polys(xi):
    out = []
    for a in range(len(xi)):
        num = Pn.fromroots([xi[b] for b in range(len(xi)) if b != a])
        out.append(num / num(xi[a]))
    return out


def integral(poly):
    F = poly.integ()
    return F(1.0) - F(-1.0)


def exact_1d(p, h, ncell, x0=None):
    """Assembled periodic 1D stiffness (2/h) int l_a' l_b', mass (h/2) int l_a l_b and,
    with x0, (h/2) int l_a l_b (x - x0)^2, by exact polynomial integration."""
    xi, _ = gll_nodes_weights(p)
    ls = lagrange_polys(xi)
    G = ncell * p
    K, Mm, V = np.zeros((G, G)), np.zeros((G, G)), np.zeros((G, G))
    for e in range(ncell):
        idx = [(e * p + a) % G for a in range(p + 1)]
        xmap = Pn([e * h + h / 2.0 - (x0 if x0 is not None else 0.0), h / 2.0])   # x(xi) - x0
        for a in range(p + 1):
            for b in range(p + 1):
                K[idx[a], idx[b]] += (2.0 / h) * integral(ls[a].deriv() * ls[b].deriv())
                Mm[idx[a], idx[b]] += (h / 2.0) * integral(ls[a] * ls[b])
                if x0 is not None:
                    V[idx[a], idx[b]] += (h / 2.0) * integral(ls[a] * ls[b] * xmap * xmap)
    return K, Mm, V


def zero_fields(mesh, nq):
    return np.zeros((mesh.ncells, nq ** 3))


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_lagrange_tables(p):
    xi, _ = gll_nodes_weights(p)
    B, D = lagrange_tables(xi, xi)
    np.testing.assert_allclose(B, np.eye(p + 1), atol=1e-13)
    np.testing.assert_allclose(D, lagrange_derivative_matrix(xi), atol=1e-11)
    x = np.linspace(-1, 1, 13)
    B, D = lagrange_tables(xi, x)
    for k in range(p + 1):
        np.testing.assert_allclose(B @ xi ** k, x ** k, atol=1e-12)
        np.testing.assert_allclose(D @ xi ** k, k * x ** max(k - 1, 0) if k else 0 * x, atol=1e-10)


def test_consistent_mass_properties():
    mesh = Mesh((2, 3, 2), (4.0, 7.5, 5.0), 3)
    Hs = {nq: FullMassHamiltonian(mesh, nq, zero_fields(mesh, nq)) for nq in (4, 5, 7)}
    M = Hs[5].Mscalar.toarray()
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    assert np.linalg.eigvalsh(M).min() > 0
    # row sums: int N_I, which GLL quadrature integrates exactly -> the GLL-integrated mass
    np.testing.assert_allclose(M.sum(axis=1), mesh.lumped_mass(), rtol=1e-13)
    assert abs(M.sum() - 4.0 * 7.5 * 5.0) < 1e-11
    # any n_q >= p + 1 integrates degree 2p exactly
    for nq in (4, 7):
        np.testing.assert_allclose(Hs[nq].Mscalar.toarray(), M, atol=1e-14)
        np.testing.assert_allclose(Hs[nq].Ke, Hs[5].Ke, atol=1e-12)
    # element mass = tensor product of the exact 1D element masses
    xi, _ = gll_nodes_weights(3)
    ls = lagrange_polys(xi)
    m1 = np.array([[integral(a * b) for b in ls] for a in ls])
    np.testing.assert_allclose(Hs[5].Me, mesh.detJ * np.kron(m1, np.kron(m1, m1)), atol=1e-14)


def test_free_electron_spectrum_is_sum_of_exact_1d_spectra():
    n, L, p = (2, 2, 3), (6.0, 6.0, 9.0), 3
    mesh = Mesh(n, L, p)
    H = FullMassHamiltonian(mesh, p + 2, zero_fields(mesh, p + 2))
    K3 = H.Hloc[0::2, 0::2].real.toarray()
    ev3 = sla.eigh(K3, H.Mscalar.toarray(), eigvals_only=True)
    ones = []
    for d in range(3):
        K1, M1, _ = exact_1d(p, L[d] / n[d], n[d])
        ones.append(sla.eigh(0.5 * K1, M1, eigvals_only=True))
    sums = np.sort((ones[0][:, None, None] + ones[1][None, :, None] + ones[2][None, None, :]).ravel())
    np.testing.assert_allclose(ev3, sums, atol=1e-9 * max(1.0, sums.max()))


def test_consistent_mass_levels_are_galerkin_upper_bounds():
    # conforming Galerkin with the exact mass: every discrete level lies above the exact one
    # (min-max), and the first plane-wave shell (2 pi / L)^2 / 2 (6 states) is approached from above
    L = 8.0
    exact = 0.5 * (2 * np.pi / L) ** 2
    errs = []
    for p in (2, 3, 4):
        mesh = Mesh(2, L, p)
        H = FullMassHamiltonian(mesh, p + 2, zero_fields(mesh, p + 2))
        ev = sla.eigh(H.Hloc[0::2, 0::2].real.toarray(), H.Mscalar.toarray(), eigvals_only=True)
        assert abs(ev[0]) < 1e-10
        shell = ev[1:7]                            # cos / sin triplets may split on coarse meshes
        assert np.all(shell >= exact - 1e-12)
        errs.append(shell.max() - exact)
    assert errs[0] > errs[1] > errs[2] > 0


def test_harmonic_oscillator_is_separable_and_exact():
    n, L, p, omega = 2, 8.0, 3, 0.6
    mesh = Mesh(n, L, p)
    nq = p + 2                                     # exact for degree 2p + 2
    H0 = FullMassHamiltonian(mesh, nq, zero_fields(mesh, nq))
    xq = H0.gauss_coords()
    V = 0.5 * omega ** 2 * np.sum((xq - L / 2) ** 2, axis=2)
    H = FullMassHamiltonian(mesh, nq, V)
    ev3 = sla.eigh(H.Hloc[0::2, 0::2].real.toarray(), H.Mscalar.toarray(), eigvals_only=True)
    K1, M1, V1 = exact_1d(p, L / n, n, x0=L / 2)
    e1 = sla.eigh(0.5 * K1 + 0.5 * omega ** 2 * V1, M1, eigvals_only=True)
    sums = np.sort((e1[:, None, None] + e1[None, :, None] + e1[None, None, :]).ravel())
    np.testing.assert_allclose(ev3, sums, atol=1e-9 * sums.max())


def _soc_problem(with_b=True):
    mesh = Mesh((2, 2, 2), 6.0, 3)
    nq = 5
    H0 = FullMassHamiltonian(mesh, nq, zero_fields(mesh, nq))
    xq = H0.gauss_coords().reshape(-1, 3)
    rng = np.random.default_rng(0)
    V = workloads.gaussian_sum_potential(xq, rng.uniform(0, 6, (3, 3)), np.array([2.0, 1.5, 1.0]),
                                         np.array([1.0, 1.2, 0.9]), np.array([6.0, 6.0, 6.0]))
    B = 0.05 * np.stack([np.cos(2 * np.pi * xq[:, 0] / 6), np.sin(2 * np.pi * xq[:, 1] / 6),
                         np.cos(2 * np.pi * xq[:, 2] / 6)]) if with_b else None
    atoms = np.array([[1.5, 1.5, 1.5], [4.5, 4.0, 4.2]])
    return FullMassHamiltonian(mesh, nq, V, B, atoms, np.array([[0.7, 0.65], [0.72, 0.6]]),
                               np.array([[0.05, 0.08], [0.03, 0.06]]))


def test_hermitian_and_kramers_pairs():
    H = _soc_problem(with_b=False)
    Hd, Md = H.dense()
    assert np.abs(Hd - Hd.conj().T).max() <= 1e-14 * np.abs(Hd).max()   # up to the rounding of the sums
    np.testing.assert_allclose(Md, Md.T, atol=1e-15 * np.abs(Md).max())
    ev = sla.eigh(Hd, Md, eigvals_only=True)
    np.testing.assert_allclose(ev[0::2], ev[1::2], atol=1e-10)
    Hb, Mb = _soc_problem(with_b=True).dense()
    eb = sla.eigh(Hb, Mb, eigvals_only=True)
    assert np.abs(eb[0::2] - eb[1::2]).max() > 1e-4       # a field splits the pairs


def test_rchfsi_with_diagonal_D_reaches_full_mass_eigenpairs_chfsi_stalls():
    H = _soc_problem()
    Hd, Md = H.dense()
    ev = sla.eigh(Hd, Md, eigvals_only=True)
    evD = sla.eigh(Hd, np.diag(H.Mdiag), eigvals_only=True)
    lmax = 1.01 * max(ev[-1], evD[-1])
    nv, nw = 16, 10
    X0 = workloads.complex_normal(3, (H.N, nv))
    _, lam, hist = rchfsi_eigensolver(H, X0, 10, lmax, 1e-9, 40, mode="rchfsi", nwanted=nw)
    assert hist[-1]["maxres"] < 1e-9
    np.testing.assert_allclose(lam[:nw], ev[:nw], atol=1e-11)
    # ChFSI with D in place of M^-1: a residual floor far above R-ChFSI's, Ritz values off
    _, lamc, histc = rchfsi_eigensolver(H, X0, 10, lmax, 1e-9, 30, mode="chfsi", nwanted=nw)
    floor = [h["maxres"] for h in histc[-10:]]
    assert min(floor) > 1e-3 and max(floor) / min(floor) < 1.01
    assert np.abs(lamc[:nw] - ev[:nw]).max() > 1e-5
    # ChFSI with the exact M^-1 converges as well (the cost R-ChFSI avoids)
    _, lame, histe = rchfsi_eigensolver(H, X0, 10, lmax, 1e-9, 40, mode="chfsi_exact_mass", nwanted=nw)
    assert histe[-1]["maxres"] < 1e-9
    np.testing.assert_allclose(lame[:nw], ev[:nw], atol=1e-11)


def test_projector_moments_converge_to_the_closed_form():
    # sum_I p_I (x_I - X)_i = int beta_{j,i} (x - X)_i exactly up to quadrature, since the
    # interpolant of a linear function is the function; the Gaussian moment in closed form
    # is N_j s^2 (2 pi s^2)^(3/2) (support cut at 7 s, inside the box: no wrap)
    L, s, X = 8.0, 0.5, np.array([4.0, 4.0, 4.0])
    Nj = np.sqrt(2.0 / (np.pi ** 1.5 * s ** 5))
    exact = Nj * s ** 2 * (2 * np.pi * s ** 2) ** 1.5
    errs = []
    for p in (3, 4, 5):
        mesh = Mesh(4, L, p)
        H = FullMassHamiltonian(mesh, p + 2, zero_fields(mesh, p + 2), None, X[None, :],
                                np.array([[s, s]]), np.array([[0.05, 0.08]]), rcut_factor=7.0)
        pr = H.projectors[0]
        xyz = mesh.node_coords()[pr["support"]] - X
        worst = 0.0
        for j in range(2):
            for i in range(3):
                col = pr["P"][0::2, 6 * j + 2 * i]              # spin-up column (j, i)
                assert np.array_equal(col, pr["P"][1::2, 6 * j + 2 * i + 1])
                worst = max(worst, abs(col @ xyz[:, i] - exact) / exact)
                other = (i + 1) % 3                             # odd in the other coordinate
                assert abs(col @ xyz[:, other]) < 1e-12 * exact
        errs.append(worst)
    # spectral convergence in p (measured 1.6e-3, 1.4e-4, 2.4e-5); a wrong weight or Jacobian is O(1)
    assert errs[0] > 5 * errs[1] and errs[1] > 5 * errs[2] and errs[2] < 1e-4


def test_fp32_rchfsi_with_diagonal_D_reaches_full_mass_eigenpairs():
    """Both approximations of the paper at once: FP32 recurrence products and D^-1 in place of
    M^-1.  With the residual in FP64 and the full M, Algorithm 1 still reaches the dense
    eigenvalues of (H, M) (measured: 15 cycles, 4.8e-14 Ha)."""
    from lowprec_emulation import rchfsi_filter_fp32
    from oracle import rayleigh_ritz
    from oracle.filters import residual
    H = _soc_problem()
    Hd, Md = H.dense()
    ev = sla.eigh(Hd, Md, eigvals_only=True)
    evD = sla.eigh(Hd, np.diag(H.Mdiag), eigvals_only=True)
    lmax = 1.01 * max(ev[-1], evD[-1])
    X, lam = rayleigh_ritz(H, workloads.complex_normal(3, (H.N, 16)))
    for _ in range(40):
        res = np.linalg.norm(residual(H, X, lam), axis=0)[:10].max()
        if res < 1e-9:
            break
        X, lam = rayleigh_ritz(H, rchfsi_filter_fp32(H, X, lam, float(lam.min()), float(lam.max()), lmax, 10))
    assert res < 1e-9
    np.testing.assert_allclose(lam[:10], ev[:10], atol=1e-11)
