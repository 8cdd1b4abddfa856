"""Filters, Lanczos bound, Rayleigh-Ritz and the eigensolver loop: GPU vs the FP64 oracle.

Filtered blocks are always compared from the same input X, Lambda and
bounds (eigenvectors are not unique, so the GPU is fed the oracle's state).
FP64 filters must agree to 1e-10 relative Frobenius.  The FP32 R-ChFSI
recurrence is checked against the residual-proportional error bound it
relies on (Eq. rChFSIrecurrence and the text around it): its error scales
with ||R||, while FP32 ChFSI stalls at an eps_32 floor.
"""
import numpy as np
import pytest

import workloads
from gpu_cases import Pair, rel, to_dev, to_host
from oracle import (chfsi_filter, lanczos_bounds, rayleigh_ritz, rchfsi_eigensolver, rchfsi_filter,
                    ritz_filter_values)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg1():
    """The 4^3-cell, p = 4, side 8 workload with its 2 spin-orbit atoms (8,192 DoF)."""
    w = workloads.workload("cfg1")
    pr = Pair(w.ncell, w.side, w.p, natoms=w.natoms, seed=w.seed)
    H = pr.H
    X0 = workloads.complex_normal(w.seed + 100, (H.N, w.nvec))
    X, lam = rayleigh_ritz(H, X0)
    v0 = workloads.complex_normal(w.seed + 200, H.N)
    lo, hi, *_ = lanczos_bounds(H, v0, w.lanczos)
    pr.X, pr.lam, pr.v0, pr.hi = X, lam, v0, hi
    pr.bounds = (float(lam.min()), float(lam.max()), hi)
    yield pr
    pr.close()


def _gpu_filter(pr, X, lam, bounds, q, mode, prec, block=0):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    Xd = to_dev(X)
    Yd = torch.zeros_like(Xd)
    R.rcf_filter(pr.g.ctx, pr.g.op, Xd, lam, q, bounds, mode, prec, block, Yd)
    return to_host(Yd)


def test_lanczos_matches_oracle(cfg1):
    from paper_2605_30128_gb300 import rchfsi as R
    lo, hi, *_ = lanczos_bounds(cfg1.H, cfg1.v0, 10)
    glo, ghi = R.rcf_lanczos_bounds(cfg1.g.ctx, cfg1.g.op, 10, to_dev(cfg1.v0)[0])
    assert abs(ghi - hi) < 1e-10 * abs(hi)
    assert abs(glo - lo) < 1e-9 * max(1.0, abs(lo))


@pytest.mark.parametrize("q", [1, 2, 10])
@pytest.mark.parametrize("block", [0, 12])
def test_chfsi_fp64(cfg1, q, block):
    from paper_2605_30128_gb300 import rchfsi as R
    ref = chfsi_filter(cfg1.H, cfg1.X, *cfg1.bounds, q)
    Y = _gpu_filter(cfg1, cfg1.X, cfg1.lam, cfg1.bounds, q, R.RCF_CHFSI, R.RCF_FP64, block)
    assert rel(Y, ref) < 1e-10


@pytest.mark.parametrize("q", [1, 2, 3, 10])
@pytest.mark.parametrize("block", [0, 12])
def test_rchfsi_fp64(cfg1, q, block):
    from paper_2605_30128_gb300 import rchfsi as R
    ref = rchfsi_filter(cfg1.H, cfg1.X, cfg1.lam, *cfg1.bounds, q)
    Y = _gpu_filter(cfg1, cfg1.X, cfg1.lam, cfg1.bounds, q, R.RCF_RCHFSI, R.RCF_FP64, block)
    assert rel(Y, ref) < 1e-10


def test_rchfsi_fp32_error_scales_with_residual(cfg1):
    """Near-converged input: X = exact eigen-block + delta * noise.  R-ChFSI in FP32 has an
    error proportional to ||R|| (so it shrinks with delta); ChFSI in FP32 does not."""
    from paper_2605_30128_gb300 import rchfsi as R
    H = cfg1.H
    # converge the oracle to a tight tolerance to get an (almost) exact eigen-block
    Xc, lam_c, hist = rchfsi_eigensolver(H, cfg1.X, q=10, lmax=cfg1.hi, tol=1e-11, max_cycles=80,
                                         nwanted=28)
    bounds = (float(lam_c.min()), float(lam_c.max()), cfg1.hi)
    noise = workloads.complex_normal(77, Xc.shape)
    nw = 28   # the wanted columns; the buffer columns above keep an O(1e-3) residual
    errs32, errs_df, errs_ch = [], [], []
    for delta in (1e-3, 1e-6):
        X = Xc + delta * noise / np.linalg.norm(noise) * np.linalg.norm(Xc)
        ref = rchfsi_filter(H, X, lam_c, *bounds, 10)
        y32 = _gpu_filter(cfg1, X, lam_c, bounds, 10, R.RCF_RCHFSI, R.RCF_FP32)
        ydf = _gpu_filter(cfg1, X, lam_c, bounds, 10, R.RCF_RCHFSI, R.RCF_FP32_DF)
        c32 = _gpu_filter(cfg1, X, lam_c, bounds, 10, R.RCF_CHFSI, R.RCF_FP32)
        # the filters act column by column, so the wanted columns can be checked alone
        errs32.append(rel(y32[:, :nw], ref[:, :nw]))
        errs_df.append(rel(ydf[:, :nw], ref[:, :nw]))
        errs_ch.append(rel(c32[:, :nw], ref[:, :nw]))
    for errs in (errs32, errs_df):
        assert errs[0] < 1e-6
        assert errs[1] < errs[0] * 1e-2          # residual-proportional
        assert errs[1] < 1e-9
    assert errs_ch[1] > 1e2 * errs32[1]          # plain FP32 ChFSI keeps its eps_32 floor


@pytest.fixture(params=[0, 1, 2], ids=["rr-fp64", "rr-df", "rr-tc"])
def rr_arith(request, cfg1):
    """Run with the cuBLAS FP64, the double-float and the tensor-core tall products."""
    from paper_2605_30128_gb300 import rchfsi as R
    R.rcf_set_rr_arith(cfg1.g.ctx, request.param)
    yield request.param
    R.rcf_set_rr_arith(cfg1.g.ctx, R.RCF_RR_TC)


def test_rayleigh_ritz_matches_oracle(cfg1, rr_arith):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H = cfg1.H
    Y = rchfsi_filter(H, cfg1.X, cfg1.lam, *cfg1.bounds, 10)
    Xo, th = rayleigh_ritz(H, Y)
    Yd = to_dev(Y)
    Xd = torch.zeros_like(Yd)
    gth = R.rcf_rayleigh_ritz(cfg1.g.ctx, cfg1.g.op, Yd, Xd)
    np.testing.assert_allclose(gth, th, rtol=1e-10, atol=1e-11)
    Xg = to_host(Xd)
    G = Xg.conj().T @ (H.Mdiag[:, None] * Xg)
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-11
    # same subspace: singular values of Xo^H M Xg are all 1
    s = np.linalg.svd(Xo.conj().T @ (H.Mdiag[:, None] * Xg), compute_uv=False)
    assert np.max(np.abs(s - 1.0)) < 1e-9


def test_cholqr2_and_orthonormal_rr_split(cfg1, rr_arith):
    """rcf_cholqr2 then rcf_rayleigh_ritz_orth = rcf_rayleigh_ritz: M-orthonormal output, same
    span as the input, Ritz values of the oracle's Rayleigh-Ritz."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H = cfg1.H
    Y = rchfsi_filter(H, cfg1.X, cfg1.lam, *cfg1.bounds, 10)
    Xo, th = rayleigh_ritz(H, Y)
    Yd = to_dev(Y)
    R.rcf_cholqr2(cfg1.g.ctx, cfg1.g.op, Yd)
    Q = to_host(Yd)
    G = Q.conj().T @ (H.Mdiag[:, None] * Q)
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-11
    # span preserved: Y = Q (Q^H M Y)
    C = Q.conj().T @ (H.Mdiag[:, None] * Y)
    assert rel(Q @ C, Y) < 1e-10
    Xd = torch.zeros_like(Yd)
    gth = R.rcf_rayleigh_ritz_orth(cfg1.g.ctx, cfg1.g.op, Yd, Xd)
    np.testing.assert_allclose(gth, th, rtol=1e-10, atol=1e-11)
    assert torch.equal(to_dev(Q), Yd)                     # Y not modified by the orthonormal RR
    with pytest.raises(R.RcfError):
        R.rcf_rayleigh_ritz_orth(cfg1.g.ctx, cfg1.g.op, Yd, Yd)   # X_out overlaps Y


def _gpu_loop(pr, X0, q, lmax, tol, cycles, mode, prec, nwanted):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    ctx, op = pr.g.ctx, pr.g.op
    Yd = to_dev(X0)
    Xd = torch.zeros_like(Yd)
    lam = R.rcf_rayleigh_ritz(ctx, op, Yd, Xd)
    cn = torch.zeros(X0.shape[1], dtype=torch.float64, device="cuda")
    hist = []
    for c in range(cycles):
        R.rcf_residual(ctx, op, Xd, lam, None, cn)
        res = cn.cpu().numpy()
        hist.append(res[:nwanted].max())
        if res[:nwanted].max() < tol:
            break
        bounds = (float(lam.min()), float(lam.max()), lmax)
        R.rcf_filter(ctx, op, Xd, lam, q, bounds, mode, prec, 0, Yd)
        lam = R.rcf_rayleigh_ritz(ctx, op, Yd, Xd)
    return lam, hist


def test_eigensolver_loop_reaches_oracle_eigenvalues(cfg1):
    """Algorithm 1 on the GPU (FP64 ChFSI, FP64 R-ChFSI, mixed FP32 R-ChFSI) converges to the
    oracle's eigenvalues within 1e-7 Ha; mixed FP32 ChFSI stalls at a residual floor."""
    from paper_2605_30128_gb300 import rchfsi as R
    H, nw = cfg1.H, 28
    X0 = workloads.complex_normal(cfg1.w.seed + 100, (H.N, cfg1.w.nvec))
    _, ref, _ = rchfsi_eigensolver(H, X0, q=10, lmax=cfg1.hi, tol=1e-10, max_cycles=120, nwanted=nw)
    for mode, prec in ((R.RCF_CHFSI, R.RCF_FP64), (R.RCF_RCHFSI, R.RCF_FP64), (R.RCF_RCHFSI, R.RCF_FP32),
                       (R.RCF_RCHFSI, R.RCF_FP32_DF)):
        lam, hist = _gpu_loop(cfg1, X0, 10, cfg1.hi, 1e-9, 150, mode, prec, nw)
        assert hist[-1] < 1e-9, (mode, prec, hist[-5:])
        assert np.max(np.abs(lam[:nw] - ref[:nw])) < 1e-7, (mode, prec)
    lam, hist = _gpu_loop(cfg1, X0, 10, cfg1.hi, 1e-9, 60, R.RCF_CHFSI, R.RCF_FP32, nw)
    assert min(hist) > 1e-8
    # the double-float Gram / projection GEMMs in the loop
    R.rcf_set_rr_arith(cfg1.g.ctx, R.RCF_RR_DF)
    try:
        lam, hist = _gpu_loop(cfg1, X0, 10, cfg1.hi, 1e-9, 150, R.RCF_RCHFSI, R.RCF_FP32_DF, nw)
    finally:
        R.rcf_set_rr_arith(cfg1.g.ctx, R.RCF_RR_TC)
    assert hist[-1] < 1e-9
    assert np.max(np.abs(lam[:nw] - ref[:nw])) < 1e-7


def test_three_cycles_match_oracle_per_cycle(cfg1):
    """The workload's 3 filter + Rayleigh-Ritz cycles: per cycle, from the oracle's state."""
    from paper_2605_30128_gb300 import rchfsi as R
    H = cfg1.H
    X, lam = cfg1.X, cfg1.lam
    for cycle in range(3):
        b = (float(lam.min()), float(lam.max()), cfg1.hi)
        ref = rchfsi_filter(H, X, lam, *b, 10)
        Y = _gpu_filter(cfg1, X, lam, b, 10, R.RCF_RCHFSI, R.RCF_FP64)
        assert rel(Y, ref) < 1e-10
        X, lam = rayleigh_ritz(H, ref)


def test_invalid_arguments_are_rejected(cfg1):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    Xd = to_dev(cfg1.X)
    Yd = torch.zeros_like(Xd)
    with pytest.raises(R.RcfError) as e:
        R.rcf_filter(cfg1.g.ctx, cfg1.g.op, Xd, cfg1.lam, 5, (1.0, 0.5, 2.0), 1, 0, 0, Yd)
    assert e.value.status == R.RCF_EINVAL
    with pytest.raises(R.RcfError):
        R.rcf_filter(cfg1.g.ctx, cfg1.g.op, Xd, cfg1.lam, 5, cfg1.bounds, 1, 0, 0, Xd)   # Y aliases X
    with pytest.raises(R.RcfError):
        R.rcf_filter(cfg1.g.ctx, cfg1.g.op, Xd, cfg1.lam, 0, cfg1.bounds, 1, 0, 0, Yd)   # degree 0
    # zero vectors is a no-op
    R.rcf_filter(cfg1.g.ctx, cfg1.g.op, Xd[:0], cfg1.lam[:0], 5, cfg1.bounds, 1, 0, 0, Yd[:0])
    with pytest.raises(R.RcfError) as e:
        R.rcf_filter(cfg1.g.ctx, cfg1.g.op, Xd, cfg1.lam, 5, cfg1.bounds, R.RCF_CHFSI, R.RCF_FP32_DF, 0, Yd)
    assert e.value.status == R.RCF_EINVAL                                               # no residual in ChFSI
    with pytest.raises(R.RcfError) as e:
        R.rcf_set_rr_arith(cfg1.g.ctx, 5)                                                # unknown RR arithmetic
    assert e.value.status == R.RCF_EINVAL
    with pytest.raises(R.RcfError) as e:
        R.rcf_set_step_kernel(cfg1.g.ctx, 7)                                             # unknown kernel
    assert e.value.status == R.RCF_EINVAL


def test_rchfsi_at_the_papers_degree_p7():
    """p = 7 (the paper's production degree, Section IV-B): FP64 R-ChFSI and ChFSI to 1e-10 of
    the oracle and the FP32 recurrence within its residual-proportional bound, on a 3 x 2 x 2
    cell mesh (Gx = 21: one ragged FP32 tile) with two spin-orbit atoms."""
    from paper_2605_30128_gb300 import rchfsi as R
    pr = Pair((3, 2, 2), (6.0, 4.0, 4.0), 7, natoms=2, seed=31)
    try:
        H = pr.H
        X, lam = rayleigh_ritz(H, workloads.complex_normal(50, (H.N, 6)))
        lo, hi, *_ = lanczos_bounds(H, workloads.complex_normal(51, H.N), 10)
        bounds = (float(lam.min()), float(lam.max()), hi)
        q = 8
        ref = rchfsi_filter(H, X, lam, *bounds, q)
        assert rel(_gpu_filter(pr, X, lam, bounds, q, R.RCF_RCHFSI, R.RCF_FP64), ref) < 1e-10
        refc = chfsi_filter(H, X, *bounds, q)
        assert rel(_gpu_filter(pr, X, lam, bounds, q, R.RCF_CHFSI, R.RCF_FP64), refc) < 1e-10
        # FP32 recurrence: error proportional to the residual of the start block
        from oracle.filters import residual
        rn = np.linalg.norm(residual(H, X, lam)) / np.linalg.norm(H.apply(X))
        err = rel(_gpu_filter(pr, X, lam, bounds, q, R.RCF_RCHFSI, R.RCF_FP32), ref)
        assert err < 1e-4 * max(rn, 1e-3), (err, rn)
    finally:
        pr.close()
