"""Pins for the oracle's finite-element pieces (GLL basis, mesh, kinetic and mass matrices).

Every check is against something other than the oracle's own formulas:
textbook closed forms, exact integrals, coordinate matching, and the
tensor-product structure of the free-electron problem.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import Mesh, gll_nodes_weights, lagrange_derivative_matrix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        p, x, w = (s.strip() for s in line.split("|"))
        env = {"sqrt": math.sqrt}
        rows.setdefault(int(p), []).append((eval(x, env), eval(w, env)))
    return rows


@pytest.mark.parametrize("p", [2, 3, 4])
def test_gll_closed_forms(p):
    xi, w = gll_nodes_weights(p)
    ref = np.array(_golden()[p])
    np.testing.assert_allclose(xi, ref[:, 0], atol=1e-15)
    np.testing.assert_allclose(w, ref[:, 1], rtol=1e-14)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_quadrature_exact_to_degree_2p_minus_1(p):
    xi, w = gll_nodes_weights(p)
    for k in range(2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * xi ** k) - exact) < 1e-13
    # not exact at degree 2p (it is Lobatto, not Gauss)
    k = 2 * p
    assert abs(np.sum(w * xi ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("p", range(1, 8))
def test_derivative_matrix_exact_on_polynomials(p):
    xi, _ = gll_nodes_weights(p)
    D = lagrange_derivative_matrix(xi)
    for k in range(p + 1):
        f = xi ** k
        df = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        np.testing.assert_allclose(D @ f, df, atol=1e-11 * max(1, k ** 2))


@pytest.mark.parametrize("n,L,p", [((2, 3, 1), (4.0, 6.0, 2.5), 3), (1, 3.0, 2), (4, 8.0, 4)])
def test_connectivity_matches_coordinates(n, L, p):
    m = Mesh(n, L, p)
    xyz = m.node_coords()
    q = m.quad_coords()
    Lv = np.broadcast_to(np.asarray(L, float), (3,))
    d = xyz[m.conn] - q
    d -= Lv * np.round(d / Lv)
    assert np.max(np.abs(d)) < 1e-12
    # each node is hit: interior nodes once, shared ones several times
    assert np.unique(m.conn).size == m.nnodes


def test_element_kinetic_exact_integrals():
    m = Mesh(1, (2.0, 3.0, 5.0), 4)
    Ke = m.element_kinetic()
    q = m.quad_coords()[0]
    assert np.allclose(Ke, Ke.T, atol=1e-14)
    np.testing.assert_allclose(Ke @ np.ones(m.nloc), 0.0, atol=1e-12)
    vol = 2.0 * 3.0 * 5.0
    for d in range(3):
        u = q[:, d]                                   # linear: 1/2 int |grad u|^2 = vol/2
        assert abs(u @ Ke @ u - 0.5 * vol) < 1e-11
    # u = x^2 on [0, 2]: 1/2 int (2x)^2 = 2 * (8/3) * 3 * 5 = 80 (degree 2 <= 2p - 1: exact)
    u = q[:, 0] ** 2
    assert abs(u @ Ke @ u - 80.0) < 1e-10


def test_mass_sums_to_volume():
    m = Mesh((3, 2, 2), (6.0, 4.0, 5.0), 3)
    assert abs(m.lumped_mass().sum() - 120.0) < 1e-11
    assert np.all(m.lumped_mass() > 0)


def _one_d_gen_eigs(m, d):
    K, W = m.assembled_1d(d)
    return sla.eigh(0.5 * K, np.diag(W), eigvals_only=True)


def test_free_electron_tensor_product_closed_form():
    """Free electron: K = 1/2(K1g (x) Wg (x) Wg + ...), M = Wg (x) Wg (x) Wg, so the 3D
    generalized eigenvalues are sums of 1D ones (each twice, for spin)."""
    from oracle import Hamiltonian
    m = Mesh((2, 1, 2), (4.0, 3.0, 5.0), 3)
    H = Hamiltonian(m, np.zeros((m.ncells, m.nloc)))
    lam = sla.eigh(H.dense(), np.diag(H.Mdiag), eigvals_only=True)
    ex, ey, ez = (_one_d_gen_eigs(m, d) for d in range(3))
    sums = np.sort((ex[:, None, None] + ey[None, :, None] + ez[None, None, :]).ravel())
    ref = np.sort(np.repeat(sums, 2))
    np.testing.assert_allclose(lam, ref, atol=1e-10 * max(1.0, ref.max()))


def test_free_electron_converges_to_plane_waves():
    """Lowest non-zero level -> |k|^2/2 with k = 2 pi / L, 12-fold (6 wave vectors x 2 spins).

    Four cells per direction, so that translation by one cell keeps the
    (cos, sin) pairs degenerate.  The 3D shell is checked densely at p = 2;
    the convergence in p is checked on the 1D factor, to which the 3D
    spectrum is tied exactly by the tensor-product test above."""
    from oracle import Hamiltonian
    m = Mesh(4, 8.0, 2)
    H = Hamiltonian(m, np.zeros((m.ncells, m.nloc)))
    lam = sla.eigh(H.dense(), np.diag(H.Mdiag), eigvals_only=True, subset_by_index=[0, 14])
    e1 = _one_d_gen_eigs(m, 0)
    assert np.max(np.abs(lam[:2])) < 1e-10
    np.testing.assert_allclose(lam[2:14], e1[1], rtol=1e-10)
    assert lam[14] > e1[1] + 1e-3
    target = 0.5 * (2 * np.pi / 8.0) ** 2
    errs = []
    for p in (2, 3, 4, 5):
        e = _one_d_gen_eigs(Mesh(4, 8.0, p), 0)
        assert abs(e[1] - e[2]) < 1e-12
        errs.append(abs(e[1] - target))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-6
