"""Parity at the benchmark's full size and launch configuration.

20^3 cells, p = 5 (2,000,000 complex DoF), 32 spin-orbit atoms, band blocks of 256
vectors, degree 40: the GPU filters a full 256-vector block exactly as bench.py
does, and the FP64 oracle (assembled sparse H) recomputes three of its columns
(first, middle, last) with the same recurrence; those columns are compared
element by element.  Connectivity is compared bit for bit for the 20^3 p = 5 and
p = 6 meshes.  The Hamiltonian product is compared on sampled rows (computed
one by one from the element matrices) for all 256 columns.
"""
import numpy as np
import pytest

import workloads
from gpu_cases import rel, to_dev, to_host

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

COLS = [0, 128, 255]


@pytest.fixture(scope="module")
def full():
    import torch
    from oracle import Hamiltonian, Mesh
    from paper_2605_30128_gb300 import rchfsi as R
    from paper_2605_30128_gb300.problem import GPUProblem
    w = workloads.workload("cfg3")
    prm = workloads.draw_parameters(w)
    mesh = Mesh(w.ncell, w.side, w.p)
    q = mesh.quad_coords().reshape(-1, 3)
    V = workloads.gaussian_sum_potential(q, prm["centres"], prm["depths"], prm["widths"], prm["L"])
    B = workloads.smooth_periodic_field(q, prm["kvec"], prm["amps"], prm["phases"], prm["L"], prm["bmax"])
    V = V.reshape(mesh.ncells, mesh.nloc)
    B = B.reshape(3, mesh.ncells, mesh.nloc)
    H = Hamiltonian(mesh, V, B, prm["atoms"], prm["proj_width"], prm["proj_h"])
    g = GPUProblem(w, params=prm)
    g.set_potential(V, B)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    X = torch.randn((w.block, H.N), dtype=torch.complex128, device="cuda", generator=gen)
    X /= torch.linalg.norm(X, dim=1, keepdim=True)
    v0 = torch.randn((H.N,), dtype=torch.complex128, device="cuda", generator=gen)
    lo, hi = R.rcf_lanczos_bounds(g.ctx, g.op, w.lanczos, v0)
    ritz = np.linspace(lo, lo + 0.05 * (hi - lo), w.block, endpoint=False)
    bounds = (lo - 1e-3 * abs(lo), lo + 0.05 * (hi - lo), hi)
    yield dict(w=w, H=H, g=g, X=X, ritz=ritz, bounds=bounds, mesh=mesh)
    g.close()


def test_connectivity_bit_exact_full_meshes():
    from oracle import Mesh
    from paper_2605_30128_gb300 import rchfsi as R
    ctx = R.rcf_create(0)
    for name in ("cfg3", "cfg5"):
        w = workloads.workload(name)
        m = R.rcf_mesh_create(ctx, w.ncell, w.side, w.p)
        assert np.array_equal(R.rcf_mesh_connectivity(m).astype(np.int64), Mesh(w.ncell, w.side, w.p).conn)
        R.rcf_mesh_destroy(m)
    R.rcf_destroy(ctx)


def test_apply_sampled_rows_all_columns(full):
    """H D^{-1} on all 256 columns (FP64 and FP32), 48 sampled rows per column computed by the
    oracle from the element matrices of the cells around each node."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H, g, X = full["H"], full["g"], full["X"]
    rng = np.random.default_rng(3)
    nodes = list(rng.integers(0, H.nnodes, 40))
    for pr in H.projectors[:4]:
        nodes.append(int(pr["support"][len(pr["support"]) // 2]))
    nodes += [0, H.nnodes - 1, 99, 100 * 100 * 99]          # corners and faces of the periodic box
    Xh = X.cpu().numpy().T
    Dinv = 1.0 / H.Mdiag
    ref = H.apply_rows(Xh * Dinv[:, None], nodes)
    rows = np.array([[2 * I, 2 * I + 1] for I in nodes]).ravel()
    Y = torch.empty_like(X)
    R.rcf_apply(g.ctx, g.op, R.RCF_FORM_H_DINV, X, Y, R.RCF_FP64)
    got = Y[:, torch.from_numpy(rows).cuda()].cpu().numpy().T
    assert rel(got, ref) < 1e-12
    X32 = X.to(torch.complex64)
    Y32 = torch.empty_like(X32)
    R.rcf_apply(g.ctx, g.op, R.RCF_FORM_H_DINV, X32, Y32, R.RCF_FP32)
    ref32 = H.apply_rows(X32.cpu().numpy().T.astype(np.complex128) * Dinv[:, None], nodes)
    got32 = Y32[:, torch.from_numpy(rows).cuda()].cpu().numpy().T.astype(np.complex128)
    assert rel(got32, ref32) < 2e-6


@pytest.mark.parametrize("mode", ["rchfsi", "chfsi"])
def test_filter_fp64_full_block_columns(full, mode):
    """FP64 filters (R-ChFSI and ChFSI) on the full 256-vector block at degree 40; three columns
    recomputed by the oracle, relative Frobenius error <= 1e-10."""
    import torch
    from oracle import chfsi_filter, rchfsi_filter
    from paper_2605_30128_gb300 import rchfsi as R
    w, H, g, X = full["w"], full["H"], full["g"], full["X"]
    Y = torch.empty_like(X)
    m = R.RCF_RCHFSI if mode == "rchfsi" else R.RCF_CHFSI
    R.rcf_filter(g.ctx, g.op, X, full["ritz"], w.degree, full["bounds"], m, R.RCF_FP64, w.block, Y)
    Xc = X[COLS].cpu().numpy().T
    if mode == "rchfsi":
        ref = rchfsi_filter(H, Xc, full["ritz"][COLS], *full["bounds"], w.degree)
    else:
        ref = chfsi_filter(H, Xc, *full["bounds"], w.degree)
    assert rel(Y[COLS].cpu().numpy().T, ref) < 1e-10


def test_filter_mixed_full_block_columns(full):
    """The benchmarked configuration: FP32 R-ChFSI on the full block at degree 40.  Against the
    oracle's FP64 filter of the same columns the error must stay at the FP32 level of the
    filtered residual part (random start block, so ||R|| is O(1) here)."""
    import torch
    from oracle import rchfsi_filter, ritz_filter_values
    from paper_2605_30128_gb300 import rchfsi as R
    w, H, g, X = full["w"], full["H"], full["g"], full["X"]
    Y = torch.empty_like(X)
    R.rcf_filter(g.ctx, g.op, X, full["ritz"], w.degree, full["bounds"], R.RCF_RCHFSI, R.RCF_FP32, w.block, Y)
    Xc = X[COLS].cpu().numpy().T
    lam = full["ritz"][COLS]
    ref = rchfsi_filter(H, Xc, lam, *full["bounds"], w.degree)
    Lq = ritz_filter_values(lam, *full["bounds"], w.degree)[w.degree]
    dz = ref - Xc * Lq[None, :]                  # D^{-1} Z_q: the part computed in FP32
    err = Y[COLS].cpu().numpy().T - ref
    assert np.linalg.norm(err) < 1e-5 * np.linalg.norm(dz)


def test_residual_df_sampled_rows_all_columns(full):
    """Double-float residual on all 256 columns at the benchmark size: 48 sampled rows per
    column against the oracle's rows of H X - M X Lambda, within 2^-40 of the magnitudes of
    the terms (the bound derived in test_gpu_residual_df)."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H, g, X = full["H"], full["g"], full["X"]
    lam = full["ritz"]
    rng = np.random.default_rng(4)
    nodes = list(rng.integers(0, H.nnodes, 40))
    for pr in H.projectors[:4]:
        nodes.append(int(pr["support"][len(pr["support"]) // 2]))
    nodes += [0, H.nnodes - 1, 99, 100 * 100 * 99]
    rows = np.array([[2 * I, 2 * I + 1] for I in nodes]).ravel()
    Xh = X.cpu().numpy().T
    ref = H.apply_rows(Xh, nodes) - H.Mdiag[rows, None] * Xh[rows] * lam[None, :]
    S = H.apply_rows(Xh, nodes, magnitudes=True) + H.Mdiag[rows, None] * np.abs(Xh[rows]) * np.abs(lam)[None, :]
    Rh = torch.empty(X.shape, dtype=torch.complex64, device="cuda")
    Rl = torch.empty_like(Rh)
    R.rcf_residual_df(g.ctx, g.op, X, lam, Rh, Rl)
    idx = torch.from_numpy(rows).cuda()
    got = Rh[:, idx].cpu().numpy().T.astype(np.complex128) + Rl[:, idx].cpu().numpy().T.astype(np.complex128)
    for part in (np.real, np.imag):
        assert np.all(np.abs(part(got) - part(ref)) <= 2.0 ** -40 * S)


def test_filter_mixed_df_full_block_columns(full):
    """FP32 R-ChFSI with the double-float residual on the full block: same bound as the
    FP32 filter with the FP64 residual."""
    import torch
    from oracle import rchfsi_filter, ritz_filter_values
    from paper_2605_30128_gb300 import rchfsi as R
    w, H, g, X = full["w"], full["H"], full["g"], full["X"]
    Y = torch.empty_like(X)
    R.rcf_filter(g.ctx, g.op, X, full["ritz"], w.degree, full["bounds"], R.RCF_RCHFSI, R.RCF_FP32_DF, w.block, Y)
    Xc = X[COLS].cpu().numpy().T
    lam = full["ritz"][COLS]
    ref = rchfsi_filter(H, Xc, lam, *full["bounds"], w.degree)
    Lq = ritz_filter_values(lam, *full["bounds"], w.degree)[w.degree]
    dz = ref - Xc * Lq[None, :]
    err = Y[COLS].cpu().numpy().T - ref
    assert np.linalg.norm(err) < 1e-5 * np.linalg.norm(dz)


def test_fp64_chfsi_16cubed_p6_full_block_columns():
    """The FP64 ChFSI configuration at full size: 16^3 cells, p = 6 (1,769,472 DoF), 16 atoms,
    512 vectors in one block, degree 30, bounds from 10 Lanczos steps; three columns (first,
    middle, last) recomputed by the oracle, relative Frobenius error <= 1e-10."""
    import torch
    from oracle import Hamiltonian, Mesh, chfsi_filter
    from paper_2605_30128_gb300 import rchfsi as R
    from paper_2605_30128_gb300.problem import GPUProblem
    w = workloads.workload("cfg2")
    prm = workloads.draw_parameters(w)
    mesh = Mesh(w.ncell, w.side, w.p)
    q = mesh.quad_coords().reshape(-1, 3)
    V = workloads.gaussian_sum_potential(q, prm["centres"], prm["depths"], prm["widths"], prm["L"])
    B = workloads.smooth_periodic_field(q, prm["kvec"], prm["amps"], prm["phases"], prm["L"], prm["bmax"])
    V = V.reshape(mesh.ncells, mesh.nloc)
    B = B.reshape(3, mesh.ncells, mesh.nloc)
    H = Hamiltonian(mesh, V, B, prm["atoms"], prm["proj_width"], prm["proj_h"])
    g = GPUProblem(w, params=prm)
    try:
        g.set_potential(V, B)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(7)
        X = torch.randn((w.nvec, H.N), dtype=torch.complex128, device="cuda", generator=gen)
        X /= torch.linalg.norm(X, dim=1, keepdim=True)
        v0 = torch.randn((H.N,), dtype=torch.complex128, device="cuda", generator=gen)
        lo, hi = R.rcf_lanczos_bounds(g.ctx, g.op, w.lanczos, v0)
        bounds = (lo - 1e-3 * abs(lo), lo + 0.05 * (hi - lo), hi)
        Y = torch.empty_like(X)
        R.rcf_filter(g.ctx, g.op, X, None, w.degree, bounds, R.RCF_CHFSI, R.RCF_FP64, w.block, Y)
        cols = [0, w.nvec // 2, w.nvec - 1]
        ref = chfsi_filter(H, X[cols].cpu().numpy().T, *bounds, w.degree)
        assert rel(Y[cols].cpu().numpy().T, ref) < 1e-10
    finally:
        g.close()


@pytest.mark.parametrize("arith", [0, 1, 2], ids=["rr-fp64", "rr-df", "rr-tc"])
def test_cholqr2_long_columns_orthonormal(full, arith):
    """Cholesky-QR2 of 64 columns of 2,000,000 rows (sums over 2M terms): the result is
    M-orthonormal to 1e-12 in every arithmetic of the tall products, and its span is the
    input's."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H, g, X = full["H"], full["g"], full["X"]
    R.rcf_set_rr_arith(g.ctx, arith)
    try:
        Y = X[:64].clone()
        R.rcf_cholqr2(g.ctx, g.op, Y)
    finally:
        R.rcf_set_rr_arith(g.ctx, R.RCF_RR_TC)
    m = torch.from_numpy(np.repeat(H.mass, 2)).cuda()
    G = (Y.conj() * m) @ Y.T
    assert (G - torch.eye(64, dtype=G.dtype, device="cuda")).abs().max().item() < 1e-12
    C = (Y.conj() * m) @ X[:64].T                      # X = Y (Y^H M X) within the span
    assert torch.linalg.norm(Y.T @ C - X[:64].T).item() < 1e-10 * torch.linalg.norm(X[:64]).item()
