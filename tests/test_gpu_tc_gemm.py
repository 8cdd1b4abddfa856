"""FP64-accurate products on the bf16 tensor cores (RCF_RR_TC) against exact and FP64 results.

- Integer entries (|x| <= 1000): every digit product and sum is an exact integer, so the
  tensor-core result must equal the exact product bit for bit; shapes cover ragged tiles
  (n, nz not multiples of 128), ragged windows (rows not a multiple of 512), node weights,
  the Hermitian lower-triangle Gram and the rotation in place.
- Random normal blocks: entry by entry within K 2^-53 max|row| max|column| (the splitting's
  bound: 7 digits of 8 bits after scaling each row / column by a power of two) of the exact
  product (Python fractions on small cases; numpy FP64 plus its own bound on larger ones).
- Cholesky-QR2 and Rayleigh-Ritz with RCF_RR_TC against the oracle and against the FP64 mode.
- The mixed-precision rotation (RCF_RR_MIXED, Section III-C-4): error bounded by the
  off-diagonal part at FP32 level, and Algorithm 1 with it reaching the oracle's eigenvalues.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads
from gpu_cases import Pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_30128_gb300 import rchfsi as R
    c = R.rcf_create(0)
    yield c
    R.rcf_destroy(c)


def _dev(A):
    """numpy (rows, ncol) complex -> CUDA tensor (ncol, rows) (columns contiguous)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda()


def _int_block(rng, rows, ncol, lim=1000):
    return (rng.integers(-lim, lim + 1, (rows, ncol)) + 1j * rng.integers(-lim, lim + 1, (rows, ncol))).astype(
        np.complex128)


def _inner(ctx, Y, Z, w=None, arith=2):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    C = torch.zeros((Z.shape[1], Y.shape[1]), dtype=torch.complex128, device="cuda")
    wt = None if w is None else torch.from_numpy(w).cuda()
    R.rcf_inner(ctx, _dev(Y), _dev(Z), C, wt, arith)
    return C.cpu().numpy().T


@pytest.mark.parametrize("rows,n,nz", [(1000, 5, 3), (3000, 128, 128), (4096, 200, 130), (70000, 40, 300)])
def test_inner_exact_on_integers(ctx, rows, n, nz):
    rng = np.random.default_rng(rows + n)
    Y = _int_block(rng, rows, n)
    Z = _int_block(rng, rows, nz)
    w = rng.integers(1, 9, rows // 2).astype(np.float64)
    ref = Y.conj().T @ (np.repeat(w, 2)[:, None] * Z)       # exact: |sums| < 2^53
    assert np.array_equal(_inner(ctx, Y, Z, w), ref)
    assert np.array_equal(_inner(ctx, Y, Z), Y.conj().T @ Z)


def test_rotate_exact_on_integers_and_in_place(ctx):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    rng = np.random.default_rng(5)
    for rows, n in ((300, 7), (5000, 130), (1000, 600)):
        Y = _int_block(rng, rows, n)
        Q = _int_block(rng, n, n, 100)
        ref = Y @ Q
        Yd, Qd = _dev(Y), _dev(Q)
        X = torch.zeros_like(Yd)
        R.rcf_rotate(ctx, Yd, Qd, X, R.RCF_RR_TC)
        assert np.array_equal(X.cpu().numpy().T, ref)
        R.rcf_rotate(ctx, Yd, Qd, Yd, R.RCF_RR_TC)           # in place
        assert np.array_equal(Yd.cpu().numpy().T, ref)


def _exact_inner(Y, Z):
    n, nz = Y.shape[1], Z.shape[1]
    out = np.zeros((n, nz), dtype=np.complex128)
    for i in range(n):
        for j in range(nz):
            a, b = Y[:, i], Z[:, j]
            re = sum(Fraction(x) * Fraction(y) for x, y in zip(np.concatenate([a.real, a.imag]),
                                                               np.concatenate([b.real, b.imag])))
            im = sum(Fraction(x) * Fraction(y) for x, y in zip(np.concatenate([a.real, -a.imag]),
                                                               np.concatenate([b.imag, b.real])))
            out[i, j] = float(re) + 1j * float(im)
    return out


def test_inner_accuracy_wide_range(ctx):
    """Columns with entries spread over many binades (one scaled by 1e-30, one with a 1e5 spike):
    error within K 2^-53 max|y_i| max|z_j| of the exact result."""
    rng = np.random.default_rng(11)
    rows = 3000
    Y = workloads.complex_normal(12, (rows, 5))
    Z = workloads.complex_normal(13, (rows, 4))
    Y[:, 2] *= 1e-30
    Z[:50, 1] *= 1e5
    C = _inner(ctx, Y, Z)
    ex = _exact_inner(Y, Z)
    K = 2 * rows
    mx = lambda v: max(np.abs(v.real).max(), np.abs(v.imag).max())
    bound = np.array([[K * 2.0 ** -53 * mx(Y[:, i]) * mx(Z[:, j]) for j in range(4)] for i in range(5)])
    assert np.all(np.abs(C.real - ex.real) <= bound) and np.all(np.abs(C.imag - ex.imag) <= bound)


def test_inner_and_rotate_match_fp64_at_scale(ctx):
    """2^20 rows x 64 columns: within 1e-13 of numpy's FP64 (relative to the norm of the
    product), and the FP64 mode of the same call agrees as well."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    rows, n = 1 << 20, 64
    Y = workloads.complex_normal(21, (rows, n)) / np.sqrt(rows)
    Z = workloads.complex_normal(22, (rows, n)) / np.sqrt(rows)
    ref = Y.conj().T @ Z
    tc = _inner(ctx, Y, Z)
    f64 = _inner(ctx, Y, Z, arith=0)
    assert np.abs(tc - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(f64 - ref).max() < 1e-13 * np.abs(ref).max()
    Q = workloads.complex_normal(23, (n, n))
    X = torch.zeros((n, rows), dtype=torch.complex128, device="cuda")
    R.rcf_rotate(ctx, _dev(Y), _dev(Q), X, R.RCF_RR_TC)
    refx = Y @ Q
    assert np.abs(X.cpu().numpy().T - refx).max() < 1e-13 * np.abs(refx).max()


@pytest.fixture(scope="module")
def cfg1():
    w = workloads.workload("cfg1")
    pr = Pair(w.ncell, w.side, w.p, natoms=w.natoms, seed=w.seed)
    yield pr
    pr.close()


def test_rayleigh_ritz_tc_matches_oracle_and_fp64(cfg1):
    import torch
    from oracle import rayleigh_ritz
    from paper_2605_30128_gb300 import rchfsi as R
    H = cfg1.H
    Y0 = workloads.complex_normal(31, (H.N, 32))
    Xo, lo = rayleigh_ritz(H, Y0)
    res = {}
    for arith in (R.RCF_RR_FP64, R.RCF_RR_TC):
        R.rcf_set_rr_arith(cfg1.g.ctx, arith)
        Yd = to_dev(Y0)
        X = torch.empty_like(Yd)
        res[arith] = (R.rcf_rayleigh_ritz(cfg1.g.ctx, cfg1.g.op, Yd, X), to_host(X))
    R.rcf_set_rr_arith(cfg1.g.ctx, R.RCF_RR_TC)
    lt, Xt = res[R.RCF_RR_TC]
    np.testing.assert_allclose(lt, lo, atol=1e-10 * np.abs(lo).max())
    np.testing.assert_allclose(lt, res[R.RCF_RR_FP64][0], atol=1e-11 * np.abs(lo).max())
    G = Xt.conj().T @ (H.Mdiag[:, None] * Xt)
    assert np.abs(G - np.eye(32)).max() < 1e-13
    # M-orthonormal bases of the same space: P = Xo^H M Xt is unitary
    P = Xo.conj().T @ (H.Mdiag[:, None] * Xt)
    sv = np.linalg.svd(P, compute_uv=False)
    assert sv.max() < 1 + 1e-12 and sv.min() > 1 - 1e-10


def test_cholqr2_tc_orthonormal_at_full_size():
    """2M DoF x 256 vectors (the bench's band block): Cholesky-QR2 in RCF_RR_TC gives an
    M-orthonormal block to 1e-13 (checked in FP64 by rcf_inner) spanning the input block."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    from paper_2605_30128_gb300.problem import GPUProblem
    w = workloads.workload("cfg3")
    g = GPUProblem(w, with_proj=False)
    try:
        R.rcf_set_rr_arith(g.ctx, R.RCF_RR_TC)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(7)
        Y = torch.randn((256, g.N), dtype=torch.complex128, device="cuda", generator=gen)
        Y0 = Y.clone()
        R.rcf_cholqr2(g.ctx, g.op, Y)
        mass = torch.from_numpy(R.rcf_mesh_mass(g.mesh)).cuda()
        G = torch.zeros((256, 256), dtype=torch.complex128, device="cuda")
        R.rcf_inner(g.ctx, Y, Y, G, mass, R.RCF_RR_FP64)
        err = (G.cpu() - torch.eye(256, dtype=torch.complex128)).abs().max().item()
        assert err < 1e-13, err
        # span: Y0 = Y (Y^H M Y0) exactly up to rounding
        Cm = torch.zeros((256, 256), dtype=torch.complex128, device="cuda")
        R.rcf_inner(g.ctx, Y, Y0, Cm, mass, R.RCF_RR_FP64)      # Cm[j, i] = (Y^H M Y0)(i, j)
        Rec = torch.zeros_like(Y0)
        R.rcf_rotate(g.ctx, Y, Cm, Rec, R.RCF_RR_FP64)
        assert (torch.linalg.norm(Rec - Y0) / torch.linalg.norm(Y0)).item() < 1e-12
    finally:
        g.close()


def test_mixed_rotation_error_is_fp32_level_in_the_offdiagonal_part(ctx):
    """Section III-C-4: X = Y Q_diag (FP64) + Y Q_offdiag (FP32-level).  For Q near the identity
    (a Rayleigh-Ritz rotation close to convergence) the error is bounded by the off-diagonal
    part alone: |X - Y Q| <= K 2^-21 max|y_r| max|Q_offdiag(:, j)| per entry (3 digits of 8
    bits), so the rotation's relative error falls with ||Q_offdiag||."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    rows, n = 20000, 96
    Y = workloads.complex_normal(41, (rows, n))
    E = workloads.complex_normal(42, (n, n))
    errs = []
    for eps in (1e-2, 1e-5):
        Q = np.diag(np.exp(1j * np.linspace(0, 3, n))) + eps * E
        Qo = Q - np.diag(np.diag(Q))
        X = torch.zeros((n, rows), dtype=torch.complex128, device="cuda")
        R.rcf_rotate(ctx, _dev(Y), _dev(Q), X, R.RCF_RR_MIXED)
        Xm = X.cpu().numpy().T
        ref = Y @ Q
        mxr = np.maximum(np.abs(Y.real), np.abs(Y.imag)).max(axis=1)
        mxq = np.maximum(np.abs(Qo.real), np.abs(Qo.imag)).max(axis=0)
        bound = 2 * n * 2.0 ** -21 * mxr[:, None] * mxq[None, :] + 4 * 2.0 ** -53 * np.abs(Y) * np.abs(np.diag(Q))
        assert np.all(np.abs(Xm.real - ref.real) <= bound) and np.all(np.abs(Xm.imag - ref.imag) <= bound)
        errs.append(np.linalg.norm(Xm - ref) / np.linalg.norm(ref))
        # the FP64-accurate rotation of the same Q is ~2^-50 of the result
        R.rcf_rotate(ctx, _dev(Y), _dev(Q), X, R.RCF_RR_TC)
        assert np.linalg.norm(X.cpu().numpy().T - ref) / np.linalg.norm(ref) < 1e-14
    assert errs[0] > 1e-10 and errs[1] < errs[0] * 1e-2      # proportional to ||Q_offdiag||
    with pytest.raises(R.RcfError):
        Yd = _dev(Y)
        R.rcf_rotate(ctx, Yd, _dev(np.eye(n, dtype=np.complex128)), Yd, R.RCF_RR_MIXED)   # in place refused


def test_eigensolver_loop_with_mixed_rotation_reaches_oracle(cfg1):
    """Algorithm 1 with the mixed FP32 R-ChFSI filter and the mixed-precision rotation
    (RCF_RR_MIXED) converges to residuals below 1e-9 and to the oracle's eigenvalues within
    1e-7 Ha, like the FP64 rotation: near convergence Q is nearly diagonal, so the FP32-level
    error of Y Q_offdiag is small in absolute terms (Section III-C-4)."""
    import torch
    from oracle import rchfsi_eigensolver
    from paper_2605_30128_gb300 import rchfsi as R
    H, nw = cfg1.H, 28
    X0 = workloads.complex_normal(cfg1.w.seed + 100, (H.N, cfg1.w.nvec))
    from oracle import lanczos_bounds
    _, hi, *_ = lanczos_bounds(H, workloads.complex_normal(cfg1.w.seed + 200, H.N), cfg1.w.lanczos)
    _, ref, _ = rchfsi_eigensolver(H, X0, q=10, lmax=hi, tol=1e-10, max_cycles=120, nwanted=nw)
    ctx, op = cfg1.g.ctx, cfg1.g.op
    hists = {}
    for arith in (R.RCF_RR_TC, R.RCF_RR_MIXED):
        R.rcf_set_rr_arith(ctx, arith)
        try:
            Yd = to_dev(X0)
            Xd = torch.zeros_like(Yd)
            lam = R.rcf_rayleigh_ritz(ctx, op, Yd, Xd)
            cn = torch.zeros(X0.shape[1], dtype=torch.float64, device="cuda")
            hist = []
            for c in range(150):
                R.rcf_residual(ctx, op, Xd, lam, None, cn)
                hist.append(cn.cpu().numpy()[:nw].max())
                if hist[-1] < 1e-9:
                    break
                R.rcf_filter(ctx, op, Xd, lam, 10, (float(lam.min()), float(lam.max()), hi), R.RCF_RCHFSI,
                             R.RCF_FP32, 0, Yd)
                lam = R.rcf_rayleigh_ritz(ctx, op, Yd, Xd)
        finally:
            R.rcf_set_rr_arith(ctx, R.RCF_RR_TC)
        assert hist[-1] < 1e-9, (arith, hist[-5:])
        assert np.max(np.abs(lam[:nw] - ref[:nw])) < 1e-7, arith
        hists[arith] = hist
    assert abs(len(hists[R.RCF_RR_MIXED]) - len(hists[R.RCF_RR_TC])) <= 2
