"""16-bit storage of the R-ChFSI recurrence (RCF_FP16, RCF_BF16): Z_k, Z_{k-1} and R stored as
binary16 / bfloat16 pairs, products in FP32, against the FP64 oracle.

- One step (rcf_cheb_step) on 16-bit inputs: the oracle evaluates the same step in FP64 from the
  exactly converted 16-bit inputs; the GPU result must be the 16-bit rounding of it (FP32
  arithmetic errs by ~1e-6 relative, far below half a 16-bit ulp, so all but the entries within
  that distance of a rounding boundary match exactly; >= 99 % here) without projectors, and within
  one 16-bit ulp of the magnitude scale with them (the spin-orbit add-back rounds a second time).
- The filter: its error against the oracle's FP64 filter falls with ||R|| (residual-proportional,
  the property R-ChFSI rests on).  Expected scale from the CPU emulation of 16-bit storage with exact
  arithmetic on this workload (tests/lowprec_emulation.py, pinned in tests/test_oracle_lowprec.py):
  9.8e-7 / 9.8e-10 (FP16) and 7.0e-6 / 7.0e-9 (BF16) at perturbations 1e-3 / 1e-6 of an
  eigenvector block; the bounds below allow 5x.
- The eigensolver loop reaches the oracle's eigenvalues within 1e-7 Ha (in
  test_gpu_filters.py and here for both 16-bit formats).
"""
import numpy as np
import pytest

import workloads
from gpu_cases import Pair, rel, to_dev, to_host
from oracle import lanczos_bounds, rayleigh_ritz, rchfsi_eigensolver, rchfsi_filter

pytestmark = pytest.mark.gpu

FMT = {"fp16": (3, 2.0 ** -11), "bf16": (4, 2.0 ** -8)}


def _to16(torch, Xc, fmt):
    """complex128 device (nvec, rows) -> interleaved 16-bit real tensor (nvec, 2 rows), and the exact
    complex128 value of what was stored."""
    dt = torch.float16 if fmt == "fp16" else torch.bfloat16
    inter = torch.view_as_real(Xc).reshape(Xc.shape[0], -1).to(dt)
    back = torch.view_as_complex(inter.to(torch.float64).reshape(Xc.shape[0], -1, 2).contiguous())
    return inter, back


def _from16(torch, T):
    return torch.view_as_complex(T.to(torch.float64).reshape(T.shape[0], -1, 2).contiguous())


@pytest.fixture(scope="module", params=[((5, 3, 2), (10.0, 6.0, 4.0), 5), ((7, 3, 2), (7.0, 4.5, 3.0), 3),
                                        ((4, 3, 2), (8.0, 6.0, 4.0), 6)], ids=lambda m: f"n{m[0]}-p{m[2]}")
def meshes(request):
    n, L, p = request.param
    plain = Pair(n, L, p, natoms=2, with_proj=False)
    proj = Pair(n, L, p, natoms=2)
    yield plain, proj
    plain.close()
    proj.close()


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_step_16bit_matches_rounded_oracle(meshes, fmt):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    prec, eps = FMT[fmt]
    alpha, beta, gamma = 0.37, -0.52, -0.81
    for pr, with_proj in zip(meshes, (False, True)):
        H = pr.H
        nv = 4
        Zk = to_dev(workloads.complex_normal(11, (H.N, nv)))
        Zm = to_dev(workloads.complex_normal(12, (H.N, nv)))
        Rr = to_dev(workloads.complex_normal(13, (H.N, nv)))
        g = torch.tensor([0.3, -1.1, 0.7, 2.0], dtype=torch.float64, device="cuda")
        zk, zk64 = _to16(torch, Zk, fmt)
        zm, zm64 = _to16(torch, Zm, fmt)
        rr, rr64 = _to16(torch, Rr, fmt)
        out = torch.empty_like(zk)
        R.rcf_cheb_step(pr.g.ctx, pr.g.op, R.RCF_FORM_H_DINV, prec, zk, zm, rr, alpha, beta, gamma, g, out)
        got = to_host(_from16(torch, out))
        Zk_h, Zm_h, R_h = to_host(zk64), to_host(zm64), to_host(rr64)
        ref = (alpha * H.apply(Zk_h / H.Mdiag[:, None]) + beta * Zk_h + gamma * Zm_h
               + R_h * g.cpu().numpy()[None, :])
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) <= 2 * eps * scale
        if not with_proj:
            dt = torch.float16 if fmt == "fp16" else torch.bfloat16
            r16 = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(ref.T))).to(dt).to(torch.float64)
            g16 = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(got.T)))
            assert float((r16 == g16).double().mean()) >= 0.99


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


@pytest.mark.parametrize("fmt,bound", [("fp16", 5e-6), ("bf16", 4e-5)])
def test_filter_16bit_error_scales_with_residual(cfg1, fmt, bound):
    H = cfg1.H
    Xc, lam_c, _ = rchfsi_eigensolver(H, cfg1.X, q=10, lmax=cfg1.hi, tol=1e-11, max_cycles=80, nwanted=28)
    b = (float(lam_c.min()), float(lam_c.max()), cfg1.hi)
    noise = workloads.complex_normal(77, Xc.shape)
    errs = []
    for delta in (1e-3, 1e-6):
        X = Xc + delta * noise / np.linalg.norm(noise) * np.linalg.norm(Xc)
        ref = rchfsi_filter(H, X, lam_c, *b, 10)
        y = _gpu_filter(cfg1, X, lam_c, b, 10, FMT[fmt][0], block=12)
        errs.append(rel(y[:, :28], ref[:, :28]))
    assert errs[0] < bound
    assert errs[1] < bound * 1e-3
    assert errs[1] < errs[0] * 1e-2


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_eigensolver_16bit_reaches_oracle_eigenvalues(cfg1, fmt):
    """Algorithm 1 with the 16-bit recurrence converges to residuals below 1e-9 and to the oracle's
    eigenvalues within 1e-7 Ha, in the same number of cycles as the FP64 filter (+-2)."""
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
                     FMT[fmt][0], 0, Yd)
        lam = R.rcf_rayleigh_ritz(ctx, op, Yd, Xd)
    assert cn.cpu().numpy()[:nw].max() < 1e-9
    assert np.max(np.abs(lam[:nw] - ref[:nw])) < 1e-7
    assert abs(cyc - (len(hist_ref) - 1)) <= 2


def test_16bit_modes_rejected_for_chfsi(cfg1):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    Xd = to_dev(cfg1.X)
    Yd = torch.zeros_like(Xd)
    for prec in (R.RCF_FP16, R.RCF_BF16):
        with pytest.raises(R.RcfError) as e:
            R.rcf_filter(cfg1.g.ctx, cfg1.g.op, Xd, cfg1.lam, 5, (-1.0, 0.5, 50.0), R.RCF_CHFSI, prec, 0, Yd)
        assert e.value.status == R.RCF_EINVAL
