"""The full consistent mass with Gauss-Legendre quadrature on the GPU (Section III-A; Section
III-B-2) against the oracle's FullMassHamiltonian (oracle/fullmass.py).

- Gauss points, projector supports (bit-exact), H X in the three forms (FP64 to 1e-12, FP32 to
  2e-6), M X (1e-13), the residual H X - M X Lambda with the full M;
- the R-ChFSI filter in FP64 against the oracle's, from the same input;
- the paper's claim, on the GPU: Algorithm 1 with R-ChFSI and the diagonal D in place of M^-1
  (FP64, and the FP32 recurrence with the FP64 residual) reaches the eigenvalues of the dense
  pencil (H, M), while ChFSI with D stalls at a residual floor.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from gpu_cases import rel, to_dev, to_host
from oracle import Mesh
from oracle.filters import residual
from oracle.fullmass import FullMassHamiltonian

pytestmark = pytest.mark.gpu

NQ = 5
ATOMS = np.array([[1.5, 1.5, 1.5], [4.5, 4.0, 4.2]])
WIDTHS = np.array([[0.7, 0.65], [0.72, 0.6]])
HCOUP = np.array([[0.05, 0.08], [0.03, 0.06]])


def _fields(xq):
    rng = np.random.default_rng(0)
    V = workloads.gaussian_sum_potential(xq, rng.uniform(0, 6, (3, 3)), np.array([2.0, 1.5, 1.0]),
                                         np.array([1.0, 1.2, 0.9]), np.array([6.0, 6.0, 6.0]))
    B = 0.05 * np.stack([np.cos(2 * np.pi * xq[:, 0] / 6), np.sin(2 * np.pi * xq[:, 1] / 6),
                         np.cos(2 * np.pi * xq[:, 2] / 6)])
    return V, B


class FMPair:
    def __init__(self, ncell=2, side=6.0, p=3, nq=NQ):
        from paper_2605_30128_gb300 import rchfsi as R
        mesh = Mesh(ncell, side, p)
        H0 = FullMassHamiltonian(mesh, nq, np.zeros((mesh.ncells, nq ** 3)))
        xq = H0.gauss_coords().reshape(-1, 3)
        V, B = _fields(xq)
        self.V = V.reshape(mesh.ncells, nq ** 3)
        self.B = B.reshape(3, mesh.ncells, nq ** 3)
        self.H = FullMassHamiltonian(mesh, nq, self.V, self.B, ATOMS, WIDTHS, HCOUP)
        self.xq = xq
        self.ctx = R.rcf_create(0)
        self.mesh = R.rcf_mesh_create(self.ctx, ncell, side, p)
        self.op = R.rcf_op_create(self.ctx, self.mesh)
        R.rcf_op_set_gauss(self.ctx, self.op, nq)
        R.rcf_potential_set(self.ctx, self.op, self.V, self.B)
        R.rcf_projectors_set(self.ctx, self.op, ATOMS, WIDTHS, HCOUP)
        self.N = self.H.N
        self.ncells, self.nq = mesh.ncells, nq

    def close(self):
        from paper_2605_30128_gb300 import rchfsi as R
        R.rcf_op_destroy(self.op)
        R.rcf_mesh_destroy(self.mesh)
        R.rcf_destroy(self.ctx)


@pytest.fixture(scope="module")
def fm():
    pr = FMPair()
    yield pr
    pr.close()


def test_gauss_points_and_projector_supports(fm):
    from paper_2605_30128_gb300 import rchfsi as R
    gp = R.rcf_op_gauss_points(fm.ctx, fm.op, fm.ncells, fm.nq).reshape(-1, 3)
    np.testing.assert_allclose(gp, fm.xq, atol=1e-13)
    for a, pr in enumerate(fm.H.projectors):
        assert np.array_equal(R.rcf_projector_support(fm.op, a).astype(np.int64), pr["support"])


@pytest.mark.parametrize("form", [0, 1, 2], ids=["H", "DinvH", "HDinv"])
def test_apply_fp64_and_fp32(fm, form):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H = fm.H
    X = workloads.complex_normal(3 + form, (H.N, 4))

    def ref_of(Xr):
        if form == 0:
            return H.apply(Xr)
        if form == 1:
            return H.apply(Xr) / H.Mdiag[:, None]
        return H.apply(Xr / H.Mdiag[:, None])

    Xd = to_dev(X)
    Yd = torch.zeros_like(Xd)
    R.rcf_apply(fm.ctx, fm.op, form, Xd, Yd, R.RCF_FP64)
    ref = ref_of(X)
    Y = to_host(Yd)
    assert rel(Y, ref) < 1e-12
    assert np.abs(Y - ref).max() < 1e-11 * np.abs(ref).max()
    X32 = X.astype(np.complex64).astype(np.complex128)
    Xd32 = to_dev(X, torch.complex64)
    Yd32 = torch.zeros_like(Xd32)
    R.rcf_apply(fm.ctx, fm.op, form, Xd32, Yd32, R.RCF_FP32)
    assert rel(to_host(Yd32), ref_of(X32)) < 2e-6


def test_mass_apply_and_residual(fm):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H = fm.H
    X = workloads.complex_normal(7, (H.N, 5))
    Xd = to_dev(X)
    Md = torch.zeros_like(Xd)
    R.rcf_mass_apply(fm.ctx, fm.op, Xd, Md, R.RCF_FP64)
    ref = H.mass_apply(X)
    assert rel(to_host(Md), ref) < 1e-13
    Md32 = torch.zeros((5, H.N), dtype=torch.complex64, device="cuda")
    R.rcf_mass_apply(fm.ctx, fm.op, to_dev(X, torch.complex64), Md32, R.RCF_FP32)
    assert rel(to_host(Md32), ref) < 1e-6
    lam = np.array([-0.4, 0.1, 0.3, 1.0, 2.5])
    Rd = torch.zeros_like(Xd)
    R.rcf_residual(fm.ctx, fm.op, Xd, lam, Rd)
    assert rel(to_host(Rd), residual(H, X, lam)) < 1e-12


def test_unsupported_paths_are_refused(fm):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    X = to_dev(workloads.complex_normal(8, (fm.N, 2)))
    Y = torch.zeros_like(X)
    for fn in (lambda: R.rcf_filter(fm.ctx, fm.op, X, np.zeros(2), 4, (-1.0, 0.0, 50.0), R.RCF_RCHFSI,
                                    R.RCF_FP32_DF, 0, Y),
               lambda: R.rcf_apply_noalloc(fm.ctx, fm.op, 0, X, Y, R.RCF_FP64)):
        with pytest.raises(R.RcfError) as ei:
            fn()
        assert ei.value.status == R.RCF_ENOTSUP


@pytest.fixture(scope="module")
def spectrum(fm):
    Hd, Md = fm.H.dense()
    ev = sla.eigh(Hd, Md, eigvals_only=True)
    evD = sla.eigh(Hd, np.diag(fm.H.Mdiag), eigvals_only=True)
    return ev, 1.01 * max(ev[-1], evD[-1])


def test_rchfsi_filter_matches_oracle(fm, spectrum):
    import torch
    from oracle import rayleigh_ritz, rchfsi_filter
    from paper_2605_30128_gb300 import rchfsi as R
    H = fm.H
    _, lmax = spectrum
    X, lam = rayleigh_ritz(H, workloads.complex_normal(9, (H.N, 8)))
    bounds = (float(lam.min()), float(lam.max()), lmax)
    for q in (1, 3, 8):
        ref = rchfsi_filter(H, X, lam, *bounds, q)
        Xd = to_dev(X)
        Yd = torch.zeros_like(Xd)
        R.rcf_filter(fm.ctx, fm.op, Xd, lam, q, bounds, R.RCF_RCHFSI, R.RCF_FP64, 0, Yd)
        assert rel(to_host(Yd), ref) < 1e-10, q


def _gpu_loop(fm, X0, lmax, mode, prec, cycles, nw, tol=1e-9):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    Yd = to_dev(X0)
    Xd = torch.zeros_like(Yd)
    lam = R.rcf_rayleigh_ritz(fm.ctx, fm.op, Yd, Xd)
    cn = torch.zeros(X0.shape[1], dtype=torch.float64, device="cuda")
    hist = []
    for _ in range(cycles):
        R.rcf_residual(fm.ctx, fm.op, Xd, lam, None, cn)
        hist.append(cn.cpu().numpy()[:nw].max())
        if hist[-1] < tol:
            break
        R.rcf_filter(fm.ctx, fm.op, Xd, lam, 10, (float(lam.min()), float(lam.max()), lmax), mode, prec, 0, Yd)
        lam = R.rcf_rayleigh_ritz(fm.ctx, fm.op, Yd, Xd)
    return lam, hist


def test_rchfsi_with_diagonal_D_reaches_full_mass_eigenpairs_chfsi_stalls(fm, spectrum):
    """Section III-B-2: with D (the lumped mass) in place of M^-1, R-ChFSI reaches the dense
    eigenvalues of (H, M) to 1e-11 (FP64) and 1e-9 (FP32 recurrence with the FP64 residual),
    while ChFSI with D stalls with a residual floor above 1e-3."""
    from paper_2605_30128_gb300 import rchfsi as R
    ev, lmax = spectrum
    nv, nw = 16, 10
    X0 = workloads.complex_normal(3, (fm.N, nv))
    for prec, tol_ev in ((R.RCF_FP64, 1e-11), (R.RCF_FP32, 1e-9)):
        lam, hist = _gpu_loop(fm, X0, lmax, R.RCF_RCHFSI, prec, 60, nw)
        assert hist[-1] < 1e-9, (prec, hist[-4:])
        np.testing.assert_allclose(lam[:nw], ev[:nw], atol=tol_ev)
    lam, hist = _gpu_loop(fm, X0, lmax, R.RCF_CHFSI, R.RCF_FP64, 30, nw)
    floor = hist[-10:]
    assert min(floor) > 1e-3 and max(floor) / min(floor) < 1.01
    assert np.abs(lam[:nw] - ev[:nw]).max() > 1e-5


@pytest.mark.parametrize("ncell,side,p,nq", [
    ((3, 2, 2), (6.0, 4.0, 4.0), 2, 4),      # unequal edges
    ((8, 2, 1), (16.0, 4.0, 2.0), 5, 7),     # two x tiles (the second ragged), a single z cell
    ((1, 3, 2), (2.0, 6.0, 4.0), 7, 8),      # one x cell: a node is its own periodic image
    ((1, 2, 1), (2.0, 4.0, 2.0), 8, 9),
    ((4, 3, 2), (8.0, 6.0, 4.0), 1, 3),
], ids=lambda v: str(v))
def test_fused_forms_and_mass_across_meshes(ncell, side, p, nq):
    """The fused full-mass kernels (x-y plane pass, per-cell potential, z march with the
    combination; M X on the same kernels) against the oracle for several degrees, tile counts
    and single-cell directions, with projectors: H D^-1 and D^-1 H combined with the recurrence
    terms, in FP64 (1e-12) and FP32 (2e-6), and M X."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    mesh = Mesh(ncell, side, p)
    H0 = FullMassHamiltonian(mesh, nq, np.zeros((mesh.ncells, nq ** 3)))
    xq = H0.gauss_coords().reshape(-1, 3)
    V, B = _fields(xq)
    atoms = np.array([[0.3 * side[0], 0.5 * side[1], 0.4 * side[2]]])
    H = FullMassHamiltonian(mesh, nq, V.reshape(mesh.ncells, -1), B.reshape(3, mesh.ncells, -1), atoms,
                            WIDTHS[:1], HCOUP[:1])
    ctx = R.rcf_create(0)
    gm = R.rcf_mesh_create(ctx, ncell, side, p)
    op = R.rcf_op_create(ctx, gm)
    try:
        R.rcf_op_set_gauss(ctx, op, nq)
        R.rcf_potential_set(ctx, op, V.reshape(mesh.ncells, -1), B.reshape(3, mesh.ncells, -1))
        R.rcf_projectors_set(ctx, op, atoms, WIDTHS[:1], HCOUP[:1])
        nv = 3
        Zk = workloads.complex_normal(31, (H.N, nv))
        Zm = workloads.complex_normal(32, (H.N, nv))
        Rr = workloads.complex_normal(33, (H.N, nv))
        g = np.array([0.4, -0.9, 1.3])
        a, b, c = 0.37, -0.52, -0.81
        Dinv = 1.0 / H.Mdiag[:, None]
        for form in (R.RCF_FORM_DINV_H, R.RCF_FORM_H_DINV):
            for prec, dt, tol in ((R.RCF_FP64, torch.complex128, 1e-12), (R.RCF_FP32, torch.complex64, 2e-6)):
                cast = (lambda X: X.astype(np.complex64).astype(np.complex128)) if prec == R.RCF_FP32 else (lambda X: X)
                zk, zm, rr = cast(Zk), cast(Zm), cast(Rr)
                op_zk = Dinv * H.apply(zk) if form == R.RCF_FORM_DINV_H else H.apply(Dinv * zk)
                ref = a * op_zk + b * zk + c * zm + rr * g[None, :]
                out = torch.empty_like(to_dev(Zk, dt))
                R.rcf_cheb_step(ctx, op, form, prec, to_dev(Zk, dt), to_dev(Zm, dt), to_dev(Rr, dt), a, b, c,
                                torch.from_numpy(g).cuda(), out)
                assert rel(to_host(out), ref) < tol, (form, prec)
        Md = torch.zeros_like(to_dev(Zk))
        R.rcf_mass_apply(ctx, op, to_dev(Zk), Md, R.RCF_FP64)
        assert rel(to_host(Md), H.mass_apply(Zk)) < 1e-13
    finally:
        R.rcf_op_destroy(op)
        R.rcf_mesh_destroy(gm)
        R.rcf_destroy(ctx)


def test_bfp_stored_residual_with_the_full_mass(fm, spectrum):
    """R kept as a 12-bit BFP stream with the full mass: the step given a stream of the oracle's
    codec equals, bit for bit, the FP32 step given the decoded R; the filter matches the FP64
    recurrence on the BFP rounding of the oracle's residual (full M) within the FP32
    recurrence's own error."""
    import torch
    from lowprec_emulation import rchfsi_filter_bfp_residual, rchfsi_filter_fp32
    from oracle import rayleigh_ritz
    from oracle.bfp import bfp_decode, bfp_encode
    from paper_2605_30128_gb300 import rchfsi as R
    H = fm.H
    nv = 3
    Zk = to_dev(workloads.complex_normal(41, (H.N, nv)), torch.complex64)
    Zm = to_dev(workloads.complex_normal(42, (H.N, nv)), torch.complex64)
    Rr = workloads.complex_normal(43, (H.N, nv))
    vals = np.ascontiguousarray(Rr.T).astype(np.complex64).view(np.float32).ravel()
    s = bfp_encode(vals, 12)
    Rdec = bfp_decode(s, vals.size, 12).astype(np.float32).view(np.complex64).reshape(nv, -1)
    stream = torch.from_numpy(np.frombuffer(s.tobytes(), dtype=np.uint8).copy()).cuda()
    g = torch.tensor([0.5, -1.2, 0.8], dtype=torch.float64, device="cuda")
    for form in (R.RCF_FORM_H_DINV, R.RCF_FORM_DINV_H):
        ob, of = torch.empty_like(Zk), torch.empty_like(Zk)
        R.rcf_cheb_step(fm.ctx, fm.op, form, R.RCF_FP32_BFP12, Zk, Zm, stream, 0.3, -0.4, -0.9, g, ob)
        R.rcf_cheb_step(fm.ctx, fm.op, form, R.RCF_FP32, Zk, Zm, torch.from_numpy(Rdec).cuda(), 0.3, -0.4, -0.9,
                        g, of)
        assert torch.equal(torch.view_as_real(ob), torch.view_as_real(of))
    _, lmax = spectrum
    X, lam = rayleigh_ritz(H, workloads.complex_normal(44, (H.N, 8)))
    b = (float(lam.min()), float(lam.max()), lmax)
    Xd = to_dev(X)
    Yd = torch.zeros_like(Xd)
    R.rcf_filter(fm.ctx, fm.op, Xd, lam, 8, b, R.RCF_RCHFSI, R.RCF_FP32_BFP12, 0, Yd)
    emul = rchfsi_filter_bfp_residual(H, X, lam, *b, 8, 12)
    ref = rchfsi_filter_fp32(H, X, lam, *b, 8)
    from oracle import rchfsi_filter
    exact = rchfsi_filter(H, X, lam, *b, 8)
    e32 = rel(ref, exact)
    assert rel(to_host(Yd), emul) < 3 * e32 + 1e-12, (rel(to_host(Yd), emul), e32)
    assert rel(emul, exact) > 10 * e32      # the 12-bit storage is what separates them
