"""Failure paths of the library on the GPU, made without faulting it.

- The bounded mbarrier waits of the TMA step kernel: with the context's wait limit at 0
  every pipeline wait gives up at once, the kernel records a time-out and returns after its
  own copies have landed; the call reports RCF_ETIMEOUT and the same context then filters
  correctly once the limit is restored.
- Cholesky-QR breakdown: a Gram matrix whose second pivot is exactly zero (built from
  exactly representable entries) makes the first pass fail; the shifted pass then runs
  (seen in the number of Gram launches) and, for a full-rank block, Cholesky-QR2 finishes
  with an M-orthonormal basis of the same span; for a rank-deficient block it returns
  RCF_ENOTSPD after the shifted attempt.
- Non-finite input: NaN in V or B is refused by rcf_potential_set; NaN in a block given to
  Cholesky-QR gives RCF_ENOTSPD.
"""
import numpy as np
import pytest

import workloads
from gpu_cases import mesh_workload, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prob():
    from paper_2605_30128_gb300.problem import GPUProblem
    # 5^3 cells at p = 5: 25 nodes per direction, divisible by the TMA kernel's 25 x 5 tiles
    w = mesh_workload(5, 10.0, 5, natoms=2, seed=23)
    g = GPUProblem(w)
    yield g
    g.close()


def test_tma_wait_timeout_reports_and_context_recovers(prob):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    g = prob
    nv = 8
    X = to_dev(workloads.complex_normal(5, (g.N, nv)))
    X /= torch.linalg.norm(X, dim=1, keepdim=True)
    lo, hi = R.rcf_lanczos_bounds(g.ctx, g.op, 10, to_dev(workloads.complex_normal(6, g.N))[0])
    lam = np.linspace(lo, lo + 0.1 * (hi - lo), nv)
    bounds = (lo, lo + 0.1 * (hi - lo), hi)
    Yref = torch.empty_like(X)
    R.rcf_filter(g.ctx, g.op, X, lam, 6, bounds, R.RCF_RCHFSI, R.RCF_FP32, 0, Yref)
    R.rcf_set_step_kernel(g.ctx, R.RCF_STEP_TMA)
    try:
        Y = torch.empty_like(X)
        R.rcf_set_wait_limit(g.ctx, 0)
        with pytest.raises(R.RcfError) as ei:
            R.rcf_filter(g.ctx, g.op, X, lam, 6, bounds, R.RCF_RCHFSI, R.RCF_FP32, 0, Y)
        assert ei.value.status == R.RCF_ETIMEOUT
        R.rcf_sync(g.ctx)                        # the error word was cleared by the report
        R.rcf_set_wait_limit(g.ctx, 1 << 24)
        for _ in range(2):
            R.rcf_filter(g.ctx, g.op, X, lam, 6, bounds, R.RCF_RCHFSI, R.RCF_FP32, 0, Y)
            assert rel(to_host(Y), to_host(Yref)) < 1e-5
    finally:
        R.rcf_set_wait_limit(g.ctx, 1 << 24)
        R.rcf_set_step_kernel(g.ctx, R.RCF_STEP_CPASYNC)
    with pytest.raises(R.RcfError) as ei:
        R.rcf_set_wait_limit(g.ctx, -1)
    assert ei.value.status == R.RCF_EINVAL


def _exact_entry(m):
    """(c, v): fl(sqrt(m) * c) == v exactly, v with at most 21 significant bits (so v^2 and
    sqrt(v^2) are exact in FP64).  The Gram kernel scales row I by sqrt(M_I)."""
    r = np.sqrt(m)
    for k in range(1 << 12):
        v = 1.0 + k * 2.0 ** -20
        c = v / r
        for _ in range(4):                               # a few ulps around v / sqrt(m)
            if r * c == v:
                return c, v
            c = np.nextafter(c, np.inf if r * c < v else -np.inf)
    raise AssertionError("no exact entry found")


def _gram_launches(g, fn):
    from paper_2605_30128_gb300 import rchfsi as R
    before = R.rcf_launch_count(g.ctx)
    fn()
    return R.rcf_launch_count(g.ctx) - before


def test_cholqr_shifted_pass_engages_on_exact_breakdown(prob):
    """Run with the FP64 tall products, whose Gram matrix is one kernel plus cuBLAS per pass
    (the launch count is the observable).  Columns y1 = s e_r and y2 = s e_r + tau e_t with M_r s^2 = 1 and M_t tau^2 = 1e-18: the
    Gram matrix is v^2 [[1, 1], [1, 1]] exactly in FP64 (v^2 + 1e-18 rounds to v^2), so the first
    Cholesky factorisation meets a zero pivot.  The shifted pass makes the block well
    conditioned, the two plain passes finish: 4 Gram launches instead of 2."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    g = prob
    mass = R.rcf_mesh_mass(g.mesh)
    r, t = 17, 901
    s, _ = _exact_entry(mass[r])
    tau = np.sqrt(1e-18 / mass[t])
    Y = np.zeros((g.N, 2), dtype=np.complex128)
    Y[2 * r, :] = s
    Y[2 * t, 1] = tau
    Yd = to_dev(Y)
    # a well-conditioned block of the same size: two Gram launches
    Yok = to_dev(workloads.complex_normal(7, (g.N, 2)))
    R.rcf_set_rr_arith(g.ctx, R.RCF_RR_FP64)
    try:
        assert _gram_launches(g, lambda: R.rcf_cholqr2(g.ctx, g.op, Yok)) == 2
        assert _gram_launches(g, lambda: R.rcf_cholqr2(g.ctx, g.op, Yd)) == 4
    finally:
        R.rcf_set_rr_arith(g.ctx, R.RCF_RR_TC)
    Q = to_host(Yd)
    Md = np.repeat(mass, 2)
    G = Q.conj().T @ (Md[:, None] * Q)
    assert np.abs(G - np.eye(2)).max() < 1e-12
    # same span: the orthonormal basis reproduces e_r and e_t
    for row in (2 * r, 2 * t):
        e = np.zeros(g.N)
        e[row] = 1.0
        c = Q.conj().T @ (Md * e)
        assert abs(np.linalg.norm(Q @ c - e)) < 1e-8


def test_cholqr_rank_deficient_block_fails_after_the_shifted_pass(prob):
    from paper_2605_30128_gb300 import rchfsi as R
    g = prob
    mass = R.rcf_mesh_mass(g.mesh)
    r = 40
    Y = np.zeros((g.N, 2), dtype=np.complex128)
    Y[2 * r, :] = _exact_entry(mass[r])[0]           # two identical columns: rank 1
    Yd = to_dev(Y)
    R.rcf_set_rr_arith(g.ctx, R.RCF_RR_FP64)
    try:
        with pytest.raises(R.RcfError) as ei:
            R.rcf_cholqr2(g.ctx, g.op, Yd)
    finally:
        R.rcf_set_rr_arith(g.ctx, R.RCF_RR_TC)
    assert ei.value.status == R.RCF_ENOTSPD
    # the context stays usable
    Yok = to_dev(workloads.complex_normal(8, (g.N, 3)))
    R.rcf_cholqr2(g.ctx, g.op, Yok)


def test_nan_inputs_are_refused(prob):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    g = prob
    V = g.V.copy()
    V[3, 5] = np.nan
    with pytest.raises(R.RcfError) as ei:
        R.rcf_potential_set(g.ctx, g.op, V, g.B)
    assert ei.value.status == R.RCF_EINVAL
    B = g.B.copy()
    B[1, 0, 0] = np.inf
    with pytest.raises(R.RcfError) as ei:
        R.rcf_potential_set(g.ctx, g.op, torch.from_numpy(g.V).cuda(), torch.from_numpy(B).cuda())
    assert ei.value.status == R.RCF_EINVAL
    R.rcf_potential_set(g.ctx, g.op, g.V, g.B)        # the operator keeps working
    Y = workloads.complex_normal(9, (g.N, 3))
    Y[100, 1] = np.nan
    for arith in (R.RCF_RR_TC, R.RCF_RR_FP64, R.RCF_RR_DF):
        R.rcf_set_rr_arith(g.ctx, arith)
        try:
            with pytest.raises(R.RcfError) as ei:
                R.rcf_cholqr2(g.ctx, g.op, to_dev(Y))
        finally:
            R.rcf_set_rr_arith(g.ctx, R.RCF_RR_TC)
        assert ei.value.status == R.RCF_ENOTSPD, arith
    # a NaN or an infinity in an operand of the tensor-core products gives NaN outputs
    import torch
    Yd = to_dev(Y)
    C = torch.zeros((3, 3), dtype=torch.complex128, device="cuda")
    R.rcf_inner(g.ctx, Yd, Yd, C, None, R.RCF_RR_TC)
    Cn = C.cpu().numpy()
    assert np.isnan(Cn[1, :]).all() and np.isnan(Cn[:, 1]).all() and np.isfinite(Cn[0, 0])
    Yi = workloads.complex_normal(10, (g.N, 3))
    Yi[7, 2] = np.inf
    Q = to_dev(np.eye(3, dtype=np.complex128))
    X = torch.zeros_like(Yd)
    R.rcf_rotate(g.ctx, to_dev(Yi), Q, X, R.RCF_RR_TC)
    Xn = X.cpu().numpy()
    assert np.isnan(Xn[:, 7]).all() and np.isfinite(np.delete(Xn, 7, axis=1)).all()
