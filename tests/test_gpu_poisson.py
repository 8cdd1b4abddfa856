"""The periodic Poisson solve on the GPU (Section III-B-1; Algorithm pcg_fusion) against the
FP64 oracle (oracle/poisson.py).

- K x (rcf_laplacian) against the oracle's assembled Laplacian, entry by entry (1e-12 of the
  magnitude of the entry's terms), on meshes with p = 1 .. 8, single-cell directions and
  unequal cell edges;
- PCG with the Chebyshev-Jacobi preconditioner: the same iterates as the oracle's PCG for the
  first iterations (1e-10), the same iteration count to a tolerance, the solution of the
  oracle within 1e-9; degree 0 (Jacobi) as well; the plane-wave charge's continuum limit;
- invalid arguments rejected.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import Mesh
from oracle.poisson import chebyshev_jacobi, laplacian, pcg, poisson_rhs

pytestmark = pytest.mark.gpu

MESHES = [
    ((2, 2, 2), 6.0, 3),
    ((3, 2, 1), (6.0, 5.0, 1.5), 4),     # unequal edges, a single cell along z
    ((2, 3, 2), (4.0, 6.0, 4.0), 5),
    ((1, 2, 2), (2.0, 4.0, 4.0), 7),     # one cell along x: a node is its own periodic image
    ((2, 1, 2), (4.0, 2.0, 4.0), 8),
    ((5, 4, 3), (10.0, 8.0, 6.0), 1),
]


def _mesh_pair(ncell, side, p):
    from paper_2605_30128_gb300 import rchfsi as R
    ctx = R.rcf_create(0)
    nc = ncell if isinstance(ncell, tuple) else (ncell,) * 3
    sd = side if isinstance(side, tuple) else (side,) * 3
    gm = R.rcf_mesh_create(ctx, nc, sd, p)
    return ctx, gm, Mesh(ncell, side, p)


def _close(ctx, gm):
    from paper_2605_30128_gb300 import rchfsi as R
    R.rcf_mesh_destroy(gm)
    R.rcf_destroy(ctx)


@pytest.mark.parametrize("ncell,side,p", MESHES, ids=lambda v: str(v))
def test_laplacian_matches_oracle(ncell, side, p):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    ctx, gm, mesh = _mesh_pair(ncell, side, p)
    try:
        K = laplacian(mesh)
        x = np.random.default_rng(p).standard_normal(mesh.nnodes)
        y = torch.zeros(mesh.nnodes, dtype=torch.float64, device="cuda")
        R.rcf_laplacian(ctx, gm, torch.from_numpy(x).cuda(), y)
        ref = K @ x
        S = abs(K) @ np.abs(x)
        assert np.max(np.abs(y.cpu().numpy() - ref) / S) < 1e-12
    finally:
        _close(ctx, gm)


def _problem(ncell, side, p, seed=0):
    mesh = Mesh(ncell, side, p)
    K = laplacian(mesh)
    Kd = K.diagonal().copy()
    f = poisson_rhs(mesh, np.random.default_rng(seed).standard_normal(mesh.nnodes))
    b = 1.05 * spla.eigsh(spla.LinearOperator(K.shape, matvec=lambda v: (K @ v) / Kd), k=1, which="LM",
                          return_eigenvectors=False)[0]
    return mesh, K, Kd, f, b


@pytest.mark.parametrize("m", [0, 1, 5])
def test_pcg_iterates_match_oracle(m):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    ctx, gm, _ = _mesh_pair(3, 6.0, 4)
    try:
        mesh, K, Kd, f, b = _problem(3, 6.0, 4)
        a = b / 20.0
        pre = (lambda r: r / Kd) if m == 0 else (lambda r: chebyshev_jacobi(K, Kd, r, m, a, b))
        fd = torch.from_numpy(f).cuda()
        for k in (1, 2, 5):
            xo, ito, histo = pcg(K, f, pre, 0.0, k)
            x = torch.zeros_like(fd)
            it, res = R.rcf_poisson_pcg(ctx, gm, fd, x, m, a, b, 0.0, k)
            assert it == ito == k
            np.testing.assert_allclose(x.cpu().numpy(), xo, atol=1e-10 * np.abs(xo).max())
            assert abs(res - histo[-1]) < 1e-10 * histo[0]
        # to a tolerance: the same iteration count and solution
        xo, ito, histo = pcg(K, f, pre, 1e-10, 2000)
        x = torch.zeros_like(fd)
        it, res = R.rcf_poisson_pcg(ctx, gm, fd, x, m, a, b, 1e-10, 2000)
        assert res < 1e-10 and abs(it - ito) <= 1
        np.testing.assert_allclose(x.cpu().numpy(), xo, atol=1e-9 * np.abs(xo).max())
    finally:
        _close(ctx, gm)


def test_plane_wave_charge_continuum_limit_and_initial_guess():
    """-lap V = 4 pi cos(2 pi x / L): the GPU solution converges to 4 pi (L / 2 pi)^2 cos(2 pi x / L)
    in p; a solve started from the converged solution stops at once."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    L = 6.0
    errs = []
    for p in (2, 3, 4, 5):
        ctx, gm, mesh = _mesh_pair(2, L, p)
        try:
            K = laplacian(mesh)
            Kd = K.diagonal().copy()
            xc = mesh.node_coords()[:, 0]
            f = poisson_rhs(mesh, np.cos(2 * np.pi * xc / L))
            b = 1.05 * spla.eigsh(spla.LinearOperator(K.shape, matvec=lambda v: (K @ v) / Kd), k=1, which="LM",
                                  return_eigenvectors=False)[0]
            fd = torch.from_numpy(f).cuda()
            x = torch.zeros_like(fd)
            it, res = R.rcf_poisson_pcg(ctx, gm, fd, x, 5, b / 20.0, b, 1e-11, 500)
            assert res < 1e-11
            V = x.cpu().numpy()
            M = mesh.lumped_mass()
            V = V - (M @ V) / M.sum()
            exact = 4 * np.pi * (L / (2 * np.pi)) ** 2 * np.cos(2 * np.pi * xc / L)
            errs.append(np.abs(V - exact).max() / np.abs(exact).max())
            it2, _ = R.rcf_poisson_pcg(ctx, gm, fd, x, 5, b / 20.0, b, 1e-10, 500)
            assert it2 == 0
        finally:
            _close(ctx, gm)
    assert all(errs[i] > 3 * errs[i + 1] for i in range(3)) and errs[-1] < 1e-3


def test_invalid_arguments():
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    ctx, gm, mesh = _mesh_pair(2, 4.0, 2)
    try:
        f = torch.zeros(mesh.nnodes, dtype=torch.float64, device="cuda")
        for args in ((5, 1.0, 0.5), (5, -1.0, 2.0), (-1, 0.1, 1.0)):
            with pytest.raises(R.RcfError) as ei:
                R.rcf_poisson_pcg(ctx, gm, f, torch.zeros_like(f), args[0], args[1], args[2], 1e-8, 10)
            assert ei.value.status == R.RCF_EINVAL
        with pytest.raises(R.RcfError):
            R.rcf_poisson_pcg(ctx, gm, f, f, 3, 0.1, 1.0, 1e-8, 10)          # x overlaps f
        with pytest.raises(R.RcfError):
            R.rcf_laplacian(ctx, gm, f, f)                                     # y overlaps x
    finally:
        _close(ctx, gm)


def test_default_interval_from_the_gershgorin_bound():
    """b <= 0: the library takes the Chebyshev interval from the Gershgorin bound of
    diag(K)^-1 K; the solve converges to the oracle's solution."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    ctx, gm, _ = _mesh_pair(3, 6.0, 5)
    try:
        mesh, K, Kd, f, b = _problem(3, 6.0, 5, seed=3)
        xo, _, _ = pcg(K, f, lambda r: chebyshev_jacobi(K, Kd, r, 5, b / 20.0, b), 1e-11, 2000)
        fd = torch.from_numpy(f).cuda()
        x = torch.zeros_like(fd)
        it, res = R.rcf_poisson_pcg(ctx, gm, fd, x, 5, 0.0, 0.0, 1e-11, 2000)
        assert res < 1e-11 and it > 0
        np.testing.assert_allclose(x.cpu().numpy(), xo, atol=1e-9 * np.abs(xo).max())
    finally:
        _close(ctx, gm)
