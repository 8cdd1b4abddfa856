"""R kept as a 12-bit block floating-point stream inside the FP32 recurrence (RCF_FP32_BFP12;
Section III-C-3's format, one block per node 4-tuple and vector) against the oracle.

- One step (rcf_cheb_step) with R given as a stream that the oracle's codec wrote: bit for bit the
  same as the FP32 step given the decoded R as complex64 (the kernel's decode is exact), and within
  the FP32 rounding of the FP64 evaluation of the step with the decoded R, on meshes with ragged
  tiles, with and without the spin-orbit projectors.
- The filter: within the FP32 recurrence error of the FP64 recurrence run on the BFP rounding of the
  oracle's residual (tests/lowprec_emulation.py), and its error against the exact oracle filter
  falls with ||R|| (4.4e-6 at a 1e-3 perturbation on the CPU emulation, pinned in
  tests/test_oracle_lowprec.py).
- Algorithm 1 with it reaches the oracle's eigenvalues within 1e-7 Ha.
- Rejections: ChFSI, rcf_apply, a misaligned stream.
"""
import numpy as np
import pytest

import workloads
from gpu_cases import Pair, rel, to_dev, to_host
from oracle import lanczos_bounds, rayleigh_ritz, rchfsi_eigensolver, rchfsi_filter
from oracle.bfp import bfp_decode, bfp_encode

pytestmark = pytest.mark.gpu


def _stream_of(torch, R64):
    """(device stream, decoded complex128 host block) of the complex (N, nvec) block R64: its FP32
    rounding encoded by the oracle's codec, node 4-tuples column after column."""
    vals = np.ascontiguousarray(R64.T).astype(np.complex64).view(np.float32).ravel()
    s = bfp_encode(vals, 12)
    dec = bfp_decode(s, vals.size, 12).astype(np.float32).view(np.complex64).reshape(R64.shape[1], -1).T
    return torch.from_numpy(np.frombuffer(s.tobytes(), dtype=np.uint8).copy()).cuda(), dec.astype(np.complex128)


def _abs_apply(H, A):
    """|H| A for a nonnegative block A: the magnitudes of the terms of each entry of H A."""
    S = abs(H.Hloc) @ A
    for pr in H.projectors:
        S[pr["rows"]] += np.abs(pr["P"]) @ (np.abs(pr["Delta"]) @ (np.abs(pr["P"]).T @ A[pr["rows"]]))
    return S


@pytest.fixture(scope="module", params=[((5, 3, 2), (10.0, 6.0, 4.0), 5), ((7, 3, 2), (7.0, 4.5, 3.0), 3),
                                        ((3, 2, 2), (6.0, 4.0, 4.0), 7)], ids=lambda m: f"n{m[0]}-p{m[2]}")
def meshes(request):
    n, L, p = request.param
    plain = Pair(n, L, p, natoms=2, with_proj=False)
    proj = Pair(n, L, p, natoms=2)
    yield plain, proj
    plain.close()
    proj.close()


def test_step_with_bfp_residual(meshes):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    alpha, beta, gamma = 0.37, -0.52, -0.81
    for pr in meshes:
        H = pr.H
        nv = 5
        Zk = workloads.complex_normal(21, (H.N, nv)).astype(np.complex64).astype(np.complex128)
        Zm = workloads.complex_normal(22, (H.N, nv)).astype(np.complex64).astype(np.complex128)
        Rr = workloads.complex_normal(23, (H.N, nv)) * np.logspace(-3, 2, nv)[None, :]
        Rr[:40] = 0.0                                          # all-zero blocks
        stream, Rdec = _stream_of(torch, Rr)
        g = torch.tensor([0.3, -1.1, 0.7, 2.0, -0.05], dtype=torch.float64, device="cuda")
        zk, zm = to_dev(Zk, torch.complex64), to_dev(Zm, torch.complex64)
        out_b = torch.empty_like(zk)
        R.rcf_cheb_step(pr.g.ctx, pr.g.op, R.RCF_FORM_H_DINV, R.RCF_FP32_BFP12, zk, zm, stream,
                        alpha, beta, gamma, g, out_b)
        out_f = torch.empty_like(zk)
        R.rcf_cheb_step(pr.g.ctx, pr.g.op, R.RCF_FORM_H_DINV, R.RCF_FP32, zk, zm, to_dev(Rdec, torch.complex64),
                        alpha, beta, gamma, g, out_f)
        assert torch.equal(torch.view_as_real(out_b), torch.view_as_real(out_f))
        ref = alpha * H.apply(Zk / H.Mdiag[:, None]) + beta * Zk + gamma * Zm + Rdec * g.cpu().numpy()[None, :]
        S = (abs(alpha) * _abs_apply(H, np.abs(Zk) / H.Mdiag[:, None]) + abs(beta) * np.abs(Zk)
             + abs(gamma) * np.abs(Zm) + np.abs(Rdec) * np.abs(g.cpu().numpy())[None, :])
        got = to_host(out_b)
        assert np.max(np.abs(got - ref) / np.maximum(S, 1e-30)) < 64 * 2.0 ** -24
        # in place over Zkm1, as the filter runs it
        R.rcf_cheb_step(pr.g.ctx, pr.g.op, R.RCF_FORM_H_DINV, R.RCF_FP32_BFP12, zk, zm, stream,
                        alpha, beta, gamma, g, zm)
        assert torch.equal(torch.view_as_real(zm), torch.view_as_real(out_b))


@pytest.fixture(scope="module")
def cfg1():
    w = workloads.workload("cfg1")
    pr = Pair(w.ncell, w.side, w.p, natoms=w.natoms, seed=w.seed)
    H = pr.H
    X0 = workloads.complex_normal(w.seed + 100, (H.N, w.nvec))
    X, lam = rayleigh_ritz(H, X0)
    v0 = workloads.complex_normal(w.seed + 200, H.N)
    lo, hi, *_ = lanczos_bounds(H, v0, w.lanczos)
    pr.X0, pr.X, pr.lam, pr.hi = X0, X, lam, hi
    yield pr
    pr.close()


def _gpu_filter(pr, X, lam, bounds, q, prec, block=0):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    Xd = to_dev(X)
    Yd = torch.zeros_like(Xd)
    R.rcf_filter(pr.g.ctx, pr.g.op, Xd, lam, q, bounds, R.RCF_RCHFSI, prec, block, Yd)
    return to_host(Yd)


def test_filter_with_bfp_residual(cfg1):
    from lowprec_emulation import rchfsi_filter_bfp_residual
    from paper_2605_30128_gb300 import rchfsi as R
    H, nw = cfg1.H, 28
    Xc, lam_c, _ = rchfsi_eigensolver(H, cfg1.X, q=10, lmax=cfg1.hi, tol=1e-11, max_cycles=80, nwanted=nw)
    b = (float(lam_c.min()), float(lam_c.max()), cfg1.hi)
    noise = workloads.complex_normal(77, Xc.shape)
    errs, errs_emul, errs32 = [], [], []
    for delta in (1e-3, 1e-6):
        X = Xc + delta * noise / np.linalg.norm(noise) * np.linalg.norm(Xc)
        ref = rchfsi_filter(H, X, lam_c, *b, 10)
        emul = rchfsi_filter_bfp_residual(H, X, lam_c, *b, 10, 12)
        for block in (0, 12):
            y = _gpu_filter(cfg1, X, lam_c, b, 10, R.RCF_FP32_BFP12, block)
            errs_emul.append(rel(y[:, :nw], emul[:, :nw]))
        errs.append(rel(y[:, :nw], ref[:, :nw]))
        y32 = _gpu_filter(cfg1, X, lam_c, b, 10, R.RCF_FP32)
        errs32.append(rel(y32[:, :nw], ref[:, :nw]))
    # the storage rounding is realised exactly: what remains is the FP32 recurrence's error
    for e_em, e32 in zip(errs_emul, (errs32[0], errs32[0], errs32[1], errs32[1])):
        assert e_em < 3 * e32 + 1e-12, (errs_emul, errs32)
    assert 2e-6 < errs[0] < 9e-6
    assert 0.5e-3 < errs[1] / errs[0] < 2e-3


def test_eigensolver_with_bfp_residual_reaches_oracle_eigenvalues(cfg1):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    H, nw = cfg1.H, 28
    _, ref, hist_ref = rchfsi_eigensolver(H, cfg1.X0, q=10, lmax=cfg1.hi, tol=1e-9, max_cycles=200, nwanted=nw)
    ctx, op = cfg1.g.ctx, cfg1.g.op
    Yd = to_dev(cfg1.X0)
    Xd = torch.zeros_like(Yd)
    lam = R.rcf_rayleigh_ritz(ctx, op, Yd, Xd)
    cn = torch.zeros(Xd.shape[0], dtype=torch.float64, device="cuda")
    for cyc in range(200):
        R.rcf_residual(ctx, op, Xd, lam, None, cn)
        if cn.cpu().numpy()[:nw].max() < 1e-9:
            break
        R.rcf_filter(ctx, op, Xd, lam, 10, (float(lam.min()), float(lam.max()), cfg1.hi), R.RCF_RCHFSI,
                     R.RCF_FP32_BFP12, 0, Yd)
        lam = R.rcf_rayleigh_ritz(ctx, op, Yd, Xd)
    assert cn.cpu().numpy()[:nw].max() < 1e-9
    assert np.max(np.abs(lam[:nw] - ref[:nw])) < 1e-7
    assert abs(cyc - (len(hist_ref) - 1)) <= 2


def test_bfp_residual_rejections(cfg1):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    ctx, op = cfg1.g.ctx, cfg1.g.op
    Xd = to_dev(cfg1.X)
    Yd = torch.zeros_like(Xd)
    with pytest.raises(R.RcfError) as e:
        R.rcf_filter(ctx, op, Xd, cfg1.lam, 5, (-1.0, 0.5, 50.0), R.RCF_CHFSI, R.RCF_FP32_BFP12, 0, Yd)
    assert e.value.status == R.RCF_EINVAL
    z = to_dev(cfg1.X[:, :2], torch.complex64)
    with pytest.raises(R.RcfError) as e:
        R.rcf_apply(ctx, op, R.RCF_FORM_H, z, torch.empty_like(z), R.RCF_FP32_BFP12)
    assert e.value.status == R.RCF_EINVAL
    stream = torch.zeros(6 * (cfg1.H.N // 2) * 2 + 8, dtype=torch.uint8, device="cuda")
    g = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RcfError) as e:
        R.rcf_cheb_step(ctx, op, R.RCF_FORM_H_DINV, R.RCF_FP32_BFP12, z, None, stream[2:], 1.0, 0.0, 0.0, g,
                        torch.empty_like(z))
    assert e.value.status == R.RCF_EINVAL
    # a zero stream decodes to R = 0: the step is then the plain product
    out = torch.empty_like(z)
    R.rcf_cheb_step(ctx, op, R.RCF_FORM_H_DINV, R.RCF_FP32_BFP12, z, None, stream, 1.0, 0.0, 0.0, g, out)
    ref = torch.empty_like(z)
    R.rcf_cheb_step(ctx, op, R.RCF_FORM_H_DINV, R.RCF_FP32, z, None, None, 1.0, 0.0, 0.0, None, ref)
    assert torch.equal(torch.view_as_real(out), torch.view_as_real(ref))
