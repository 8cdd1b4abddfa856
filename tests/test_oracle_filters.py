"""Pins for the oracle's filters, Lanczos bound, Cholesky-QR / Rayleigh-Ritz and Algorithm 1."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import (chebyshev_filter_closed_form, chfsi_filter, cholqr2, filter_scalars,
                    lanczos_bounds, rayleigh_ritz, rchfsi_eigensolver, rchfsi_filter,
                    ritz_filter_values)
from oracle_cases import build_oracle, small_workload


def test_scalar_recurrence_matches_closed_form():
    lam = np.linspace(-3.0, 40.0, 57)
    lmin, lT, lmax = -2.5, 1.3, 37.0
    q = 25
    Lk = ritz_filter_values(lam, lmin, lT, lmax, q)
    for k in range(q + 1):
        ref = chebyshev_filter_closed_form(lam, lmin, lT, lmax, k)
        np.testing.assert_allclose(Lk[k], ref, rtol=1e-11, atol=1e-12)
    # normalised at lambda_min, bounded by 1/|T_k(t0)| on [lT, lmax]
    np.testing.assert_allclose(ritz_filter_values([lmin], lmin, lT, lmax, q)[:, 0], 1.0, rtol=1e-13)
    inside = (lam >= lT) & (lam <= lmax)
    c, e, _ = filter_scalars(lmin, lT, lmax, q)
    t0 = (lmin - c) / e
    Tq_t0 = np.cosh(q * np.arccosh(-t0))          # |T_q(t0)| for t0 < -1
    assert np.all(np.abs(Lk[q][inside]) <= 1.0 / Tq_t0 * (1 + 1e-9))


@pytest.fixture(scope="module")
def tiny():
    H, prm, V, B = build_oracle(small_workload(ncell=2, side=6.0, p=2))
    Hd = H.dense()
    lam, U = sla.eigh(Hd, np.diag(H.Mdiag))
    return H, lam, U


def test_filters_on_exact_eigenvectors(tiny):
    """Y_q = X C_q(Lambda) when X holds exact eigenvectors (closed form), for both filters."""
    H, lam, U = tiny
    idx = np.array([0, 3, 7, 11, 20])
    X = U[:, idx]
    lmin, lT, lmax = lam[0] - 0.1, lam[25], lam[-1] + 0.5
    q = 9
    ref = X * chebyshev_filter_closed_form(lam[idx], lmin, lT, lmax, q)[None, :]
    Y1 = chfsi_filter(H, X, lmin, lT, lmax, q)
    Y2 = rchfsi_filter(H, X, lam[idx], lmin, lT, lmax, q)
    scale = np.linalg.norm(ref)
    assert np.linalg.norm(Y1 - ref) < 1e-11 * scale
    assert np.linalg.norm(Y2 - ref) < 1e-11 * scale


def test_rchfsi_equals_chfsi_when_D_is_M(tiny):
    """Z_k := M (Y_k - X Lambda_k) satisfies the residual recurrence, so the two agree for any X, Lambda."""
    H, lam, _ = tiny
    X = workloads.complex_normal(3, (H.N, 6))
    L = np.array([-1.0, -0.5, 0.1, 0.2, 0.9, 1.4])
    lmin, lT, lmax = -1.2, 1.5, lam[-1] + 1.0
    for q in (1, 2, 7):
        Y1 = chfsi_filter(H, X, lmin, lT, lmax, q)
        Y2 = rchfsi_filter(H, X, L, lmin, lT, lmax, q)
        assert np.linalg.norm(Y1 - Y2) < 1e-12 * np.linalg.norm(Y1)
    # with D != M the two differ (the residual form is then a different method)
    Y3 = rchfsi_filter(H, X, L, lmin, lT, lmax, 7, Ddiag=H.Mdiag * 1.1)
    assert np.linalg.norm(Y3 - chfsi_filter(H, X, lmin, lT, lmax, 7)) > 1e-3 * np.linalg.norm(Y3)


def test_lanczos_bound_and_full_run(tiny):
    H, lam, _ = tiny
    v0 = workloads.complex_normal(11, H.N)
    lo, hi, al, be = lanczos_bounds(H, v0, 10)
    assert hi >= lam[-1] - 1e-9
    assert lo >= lam[0] - 1e-9
    # n steps on a small operator: the Ritz values are the eigenvalues (up to loss of orthogonality,
    # which only duplicates values); check the extremes
    lo2, hi2, al2, be2 = lanczos_bounds(H, v0, 60)
    T = np.diag(al2) + np.diag(be2[:-1], 1) + np.diag(be2[:-1], -1)
    th = np.linalg.eigvalsh(T)
    assert abs(th.max() - lam[-1]) < 1e-6 * abs(lam[-1])


def test_cholqr2_and_rayleigh_ritz(tiny):
    H, lam, _ = tiny
    Y = workloads.complex_normal(5, (H.N, 8))
    Yo = cholqr2(Y, H.Mdiag)
    G = Yo.conj().T @ (H.Mdiag[:, None] * Yo)
    assert np.max(np.abs(G - np.eye(8))) < 1e-13
    # same span: projection of Y onto span(Yo) reproduces Y
    coef = Yo.conj().T @ (H.Mdiag[:, None] * Y)
    assert np.linalg.norm(Yo @ coef - Y) < 1e-12 * np.linalg.norm(Y)
    X, th = rayleigh_ritz(H, Y)
    A = Y.conj().T @ H.apply(Y)
    S = Y.conj().T @ (H.Mdiag[:, None] * Y)
    ref = sla.eigh(0.5 * (A + A.conj().T), 0.5 * (S + S.conj().T), eigvals_only=True)
    np.testing.assert_allclose(th, ref, rtol=1e-11, atol=1e-12)
    # Ritz vectors: M-orthonormal, and X^H H X = diag(theta)
    assert np.max(np.abs(X.conj().T @ H.apply(X) - np.diag(th))) < 1e-11 * np.abs(th).max()


def test_algorithm1_converges_to_brute_force(tiny):
    H, lam, _ = tiny
    nvec = 16
    X0 = workloads.complex_normal(9, (H.N, nvec))
    lo, hi, *_ = lanczos_bounds(H, workloads.complex_normal(10, H.N), 10)
    nconv = nvec - max(4, nvec // 10)
    X, th, hist = rchfsi_eigensolver(H, X0, q=12, lmax=hi, tol=1e-9, max_cycles=60, nwanted=nconv)
    assert hist[-1]["maxres"] < 1e-9
    assert np.max(np.abs(th[:nconv] - lam[:nconv])) < 1e-9
    # ChFSI with D = M reaches the same values
    X2, th2, hist2 = rchfsi_eigensolver(H, X0, q=12, lmax=hi, tol=1e-9, max_cycles=60, mode="chfsi",
                                       nwanted=nconv)
    assert np.max(np.abs(th2[:nconv] - lam[:nconv])) < 1e-9
