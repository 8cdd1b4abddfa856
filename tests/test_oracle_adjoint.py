"""Pins for the oracle's reverse-mode filter derivative: central finite differences and a
directional (dot-product) test on a small mesh with B and spin-orbit projectors."""
import numpy as np
import pytest

import workloads
from oracle import Hamiltonian, lanczos_bounds, rayleigh_ritz, rchfsi_filter, rchfsi_filter_adjoint
from oracle import ritz_loss_head
from oracle_cases import build_oracle, small_workload


@pytest.fixture(scope="module")
def problem():
    w = small_workload(ncell=2, side=6.0, p=2)
    H, prm, V, B = build_oracle(w)
    X0 = workloads.complex_normal(21, (H.N, 8))
    X, lam = rayleigh_ritz(H, X0)
    lo, hi, *_ = lanczos_bounds(H, workloads.complex_normal(22, H.N), 10)
    bounds = (float(lam.min()), float(lam.max()), hi)
    G = workloads.complex_normal(23, (H.N, 8))
    G /= np.linalg.norm(G)
    return dict(H=H, prm=prm, V=V, B=B, X=X, lam=lam, bounds=bounds, G=G, q=6, nlow=4)


def _loss(pb, V, B, h):
    H0 = pb["H"]
    H = Hamiltonian(H0.mesh, V, B, pb["prm"]["atoms"], pb["prm"]["proj_width"], h)
    Y = rchfsi_filter(H, pb["X"], pb["lam"], *pb["bounds"], pb["q"])
    L, _, _ = ritz_loss_head(H, Y, pb["G"], pb["nlow"])
    return L


def _grad(pb):
    H = pb["H"]
    Y = rchfsi_filter(H, pb["X"], pb["lam"], *pb["bounds"], pb["q"])
    L, Ybar, direct = ritz_loss_head(H, Y, pb["G"], pb["nlow"])
    (gV, gB, gh), _ = rchfsi_filter_adjoint(H, pb["X"], pb["lam"], *pb["bounds"], pb["q"], Ybar)
    gV = gV + direct[0]
    gB = gB + direct[1]
    gh = gh + direct[2]
    dV = H.node_to_quadrature(gV)
    dB = np.stack([H.node_to_quadrature(gB[d]) for d in range(3)])
    return L, dV, dB, gh


def test_adjoint_matches_central_differences(problem):
    pb = problem
    L0, dV, dB, dh = _grad(pb)
    rng = np.random.default_rng(5)
    step = 1e-5
    V, B, h = pb["V"], pb["B"], pb["prm"]["proj_h"]
    errs = []
    for _ in range(6):
        e, l = rng.integers(V.shape[0]), rng.integers(V.shape[1])
        Vp, Vm = V.copy(), V.copy()
        Vp[e, l] += step
        Vm[e, l] -= step
        fd = (_loss(pb, Vp, B, h) - _loss(pb, Vm, B, h)) / (2 * step)
        errs.append((fd, dV[e, l]))
    for _ in range(6):
        d, e, l = rng.integers(3), rng.integers(V.shape[0]), rng.integers(V.shape[1])
        Bp, Bm = B.copy(), B.copy()
        Bp[d, e, l] += step
        Bm[d, e, l] -= step
        fd = (_loss(pb, V, Bp, h) - _loss(pb, V, Bm, h)) / (2 * step)
        errs.append((fd, dB[d, e, l]))
    for a in range(h.shape[0]):
        for j in range(2):
            hp, hm = h.copy(), h.copy()
            hp[a, j] += step
            hm[a, j] -= step
            fd = (_loss(pb, V, B, hp) - _loss(pb, V, B, hm)) / (2 * step)
            errs.append((fd, dh[a, j]))
    fd = np.array([x for x, _ in errs])
    an = np.array([y for _, y in errs])
    assert np.linalg.norm(fd - an) < 1e-7 * np.linalg.norm(fd)
    assert np.all(np.abs(fd) > 0)


def test_adjoint_directional_derivative(problem):
    pb = problem
    L0, dV, dB, dh = _grad(pb)
    rng = np.random.default_rng(8)
    pV = rng.normal(size=dV.shape)
    pB = rng.normal(size=dB.shape)
    ph = rng.normal(size=dh.shape) * 0.01
    step = 1e-5
    V, B, h = pb["V"], pb["B"], pb["prm"]["proj_h"]
    fd = (_loss(pb, V + step * pV, B + step * pB, h + step * ph)
          - _loss(pb, V - step * pV, B - step * pB, h - step * ph)) / (2 * step)
    an = np.sum(dV * pV) + np.sum(dB * pB) + np.sum(dh * ph)
    assert abs(fd - an) < 1e-7 * abs(fd)
