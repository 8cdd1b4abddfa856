"""GPU path (librchfsi through the C ABI) against the FP64 CPU oracle, element by element.

Meshes span several stencil tiles with a ragged tail in x and y (FP32 tiles
are 24-25 nodes wide and one element high, FP64 tiles about 8 x 8), single-cell
directions, and degrees p = 1 .. 8 (p = 7 is the paper's production degree).  Tolerances:
FP64 products 1e-12 relative (rounding of ~30-term sums); FP64 filters 1e-10 relative
Frobenius (the target for filtered blocks); FP32 products 2e-6 relative (float rounding of
the same sums, about 30 eps_32 in the worst row) and, entry by entry, 64 eps_32 times the
sum of the magnitudes of the entry's terms (|H| |X|): a bound on the rounding of sums of up
to ~50 terms with FP32 coefficients, which a wrong term at a tile seam would exceed.
"""
import numpy as np
import pytest

import workloads
from gpu_cases import Pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu

MESHES = [
    # FP32 tiles are 24-25 nodes wide and one element (at least ~5 rows) high; FP64 tiles ~8x8
    ((7, 3, 2), (7.0, 4.5, 3.0), 3),    # Gx = 21 < 24: one ragged FP32 tile, three FP64 tiles
    ((11, 3, 2), (11.0, 4.5, 3.0), 3),  # Gx = 33, Gy = 9: ragged in x and y
    ((4, 4, 4), 8.0, 4),                 # the 4^3 p=4 workload mesh
    ((5, 3, 2), (10.0, 6.0, 4.0), 5),    # p = 5, Gx = 25: one full tile in x, three in y
    ((7, 3, 2), (14.0, 6.0, 4.0), 5),    # p = 5, Gx = 35: a full and a ragged tile
    ((4, 3, 2), (8.0, 6.0, 4.0), 6),     # p = 6, Gx = 24, Gy = 18: 1 x 3 tiles
    ((5, 3, 2), (10.0, 6.0, 4.0), 6),    # p = 6, Gx = 30: ragged
    ((1, 2, 3), (2.0, 4.0, 6.0), 2),     # one cell along x: a node is its own periodic image
    ((9, 2, 1), (9.0, 2.0, 1.0), 1),     # p = 1
    ((5, 3, 2), (10.0, 6.0, 4.0), 7),    # p = 7: Gx = 35 (FP32 tiles 28 x 7: a full and a ragged
                                         # tile), Gy = 21; FP64 tiles 14 x 14
    ((4, 2, 2), (8.0, 4.0, 4.0), 8),     # p = 8: Gx = 32 (FP32 tiles 24 x 8: ragged), Gy = 16
    # meshes that the FP32 tiles divide, run with the TMA step kernel selected: one tile
    # per plane (its strips wrap onto itself) and several tiles; p = 5 (25 x 5 tiles),
    # p = 4 (24 x 8) and p = 6 (24 x 6)
    ((5, 1, 2), (10.0, 2.0, 4.0), 5, "tma"),
    ((10, 2, 2), (20.0, 4.0, 4.0), 5, "tma"),
    ((6, 2, 2), (12.0, 4.0, 4.0), 4, "tma"),
    ((4, 2, 2), (8.0, 4.0, 4.0), 6, "tma"),
]


@pytest.fixture(scope="module", params=MESHES, ids=lambda m: f"n{m[0]}-p{m[2]}" + ("-tma" if len(m) > 3 else ""))
def pair(request):
    from paper_2605_30128_gb300 import rchfsi as R
    n, L, p = request.param[:3]
    pr = Pair(n, L, p, natoms=2)
    if len(request.param) > 3:
        R.rcf_set_step_kernel(pr.g.ctx, R.RCF_STEP_TMA)
    yield pr
    pr.close()


def test_connectivity_and_mass_bit_exact(pair):
    from paper_2605_30128_gb300 import rchfsi as R
    conn = R.rcf_mesh_connectivity(pair.g.mesh)
    assert np.array_equal(conn.astype(np.int64), pair.H.mesh.conn)
    mass = R.rcf_mesh_mass(pair.g.mesh)
    np.testing.assert_allclose(mass, pair.H.mass, rtol=1e-14)
    q = R.rcf_mesh_quadrature_points(pair.g.mesh)
    np.testing.assert_allclose(q, pair.H.mesh.quad_coords(), atol=1e-13)
    for a, pj in enumerate(pair.H.projectors):
        sup = R.rcf_projector_support(pair.g.op, a)
        assert np.array_equal(sup.astype(np.int64), pj["support"])


@pytest.mark.parametrize("form", [0, 1, 2], ids=["H", "DinvH", "HDinv"])
def test_apply_fp64(pair, form):
    from paper_2605_30128_gb300 import rchfsi as R
    H = pair.H
    X = workloads.complex_normal(3, (H.N, 5))
    if form == 0:
        ref = H.apply(X)
    elif form == 1:
        ref = H.apply(X) / H.Mdiag[:, None]
    else:
        ref = H.apply(X / H.Mdiag[:, None])
    Xd = to_dev(X)
    Yd = Xd.new_zeros(Xd.shape)
    R.rcf_apply(pair.g.ctx, pair.g.op, form, Xd, Yd, R.RCF_FP64)
    Y = to_host(Yd)
    assert rel(Y, ref) < 1e-12
    assert np.max(np.abs(Y - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("form", [1, 2], ids=["DinvH", "HDinv"])
def test_apply_fp32(pair, form):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H = pair.H
    X = workloads.complex_normal(4, (H.N, 3))
    X32 = X.astype(np.complex64).astype(np.complex128)
    ref = H.apply(X32) / H.Mdiag[:, None] if form == 1 else H.apply(X32 / H.Mdiag[:, None])
    Xd = to_dev(X, torch.complex64)
    Yd = Xd.new_zeros(Xd.shape)
    R.rcf_apply(pair.g.ctx, pair.g.op, form, Xd, Yd, R.RCF_FP32)
    Y = to_host(Yd)
    assert rel(Y, ref) < 2e-6
    # entry by entry against the magnitudes of the terms of each entry
    A = np.abs(X32) / H.Mdiag[:, None] if form == 2 else np.abs(X32)
    S = abs(H.Hloc) @ A
    for pr in H.projectors:
        S[pr["rows"]] += np.abs(pr["P"]) @ (np.abs(pr["Delta"]) @ (np.abs(pr["P"]).T @ A[pr["rows"]]))
    if form == 1:
        S = S / H.Mdiag[:, None]
    eps32 = 2.0 ** -24
    worst = np.max(np.abs(Y - ref) / (S + 1e-300))
    assert worst < 64 * eps32, worst


def test_apply_strided_leading_dimension(pair):
    """ld > 2M: vectors inside a wider buffer."""
    from paper_2605_30128_gb300 import rchfsi as R
    H = pair.H
    X = workloads.complex_normal(5, (H.N, 3))
    ref = H.apply(X)
    t = to_dev(X)
    import torch
    big = torch.zeros((3, H.N + 6), dtype=torch.complex128, device="cuda")
    big[:, :H.N] = t
    out = torch.full((3, H.N + 10), 7.0, dtype=torch.complex128, device="cuda")
    R.rcf_apply(pair.g.ctx, pair.g.op, 0, big[:, :H.N], out[:, :H.N], R.RCF_FP64)
    assert rel(to_host(out[:, :H.N]), ref) < 1e-12
    assert torch.all(out[:, H.N:] == 7.0)   # nothing written past the rows


def test_residual(pair):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H = pair.H
    X = workloads.complex_normal(6, (H.N, 4))
    lam = np.array([-0.3, 0.1, 0.5, 2.0])
    ref = H.apply(X) - H.Mdiag[:, None] * X * lam[None, :]
    Xd = to_dev(X)
    Rd = torch.zeros_like(Xd)
    cn = torch.zeros(4, dtype=torch.float64, device="cuda")
    R.rcf_residual(pair.g.ctx, pair.g.op, Xd, lam, Rd, cn)
    assert rel(to_host(Rd), ref) < 1e-12
    np.testing.assert_allclose(cn.cpu().numpy(), np.linalg.norm(ref, axis=0), rtol=1e-12)
