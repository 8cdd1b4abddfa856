"""Adjoint of the filter on the GPU: against the oracle's reverse sweep (which stores every
forward iterate, so it checks the GPU's checkpointed recomputation), and against central
finite differences of a Ritz-value loss on the 8^3-cell adjoint workload."""
import numpy as np
import pytest

import workloads
from gpu_cases import Pair, rel, to_dev, to_host
from oracle import lanczos_bounds, rayleigh_ritz, rchfsi_filter_adjoint

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    pr = Pair((3, 2, 2), (6.0, 4.0, 4.0), 3, natoms=2, seed=17)
    H = pr.H
    X, lam = rayleigh_ritz(H, workloads.complex_normal(40, (H.N, 6)))
    lo, hi, *_ = lanczos_bounds(H, workloads.complex_normal(41, H.N), 10)
    pr.X, pr.lam = X, lam
    pr.bounds = (float(lam.min()), float(lam.max()), hi)
    pr.Ybar = workloads.complex_normal(42, (H.N, 6))
    yield pr
    pr.close()


def _gpu_adjoint(pr, q, ckpt, prec):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    dV = torch.zeros(pr.V.shape, dtype=torch.float64, device="cuda")
    dB = torch.zeros(pr.B.shape, dtype=torch.float64, device="cuda")
    dh = np.zeros((2, 2))
    R.rcf_adjoint_filter(pr.g.ctx, pr.g.op, to_dev(pr.X), pr.lam, q, pr.bounds, R.RCF_RCHFSI, prec,
                         to_dev(pr.Ybar), ckpt, dV, dB, dh)
    return dV.cpu().numpy(), dB.cpu().numpy(), dh


def _oracle_adjoint(pr, q):
    H = pr.H
    (gV, gB, gh), _ = rchfsi_filter_adjoint(H, pr.X, pr.lam, *pr.bounds, q, pr.Ybar)
    dV = H.node_to_quadrature(gV)
    dB = np.stack([H.node_to_quadrature(gB[d]) for d in range(3)])
    return dV, dB, gh


@pytest.mark.parametrize("q,ckpt", [(1, 1), (2, 1), (6, 1), (6, 2), (6, 4), (6, 10), (9, 3)])
def test_adjoint_fp64_matches_oracle(small, q, ckpt):
    from paper_2605_30128_gb300 import rchfsi as R
    gV, gB, gh = _gpu_adjoint(small, q, ckpt, R.RCF_FP64)
    oV, oB, oh = _oracle_adjoint(small, q)
    assert rel(gV, oV) < 1e-10
    assert rel(gB, oB) < 1e-10
    assert rel(gh, oh) < 1e-10


def test_adjoint_fp32_close_to_oracle(small):
    from paper_2605_30128_gb300 import rchfsi as R
    gV, gB, gh = _gpu_adjoint(small, 6, 2, R.RCF_FP32)
    oV, oB, oh = _oracle_adjoint(small, 6)
    assert rel(gV, oV) < 1e-4
    assert rel(gB, oB) < 1e-4
    assert rel(gh, oh) < 1e-4


def test_adjoint_workload_finite_differences():
    """8^3 cells, p = 4 (65,536 DoF), 4 atoms, 64 vectors, degree 15, checkpoints every 5.
    L = sum of the lowest 32 Ritz values of Y_q + Re <G, Y_q> (G seeded, scaled so both parts
    are of the same size).  Gradients by autograd (library adjoint + Ritz-value backward) vs
    central differences (step 1e-5) on 200 seeded entries of V, B and h."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    from paper_2605_30128_gb300.autograd import Operator, RChFSIFilter, RitzValues
    from paper_2605_30128_gb300.problem import GPUProblem

    w = workloads.workload("cfg4")
    g = GPUProblem(w)
    opw = Operator(g)
    N, nv, q = g.N, w.nvec, w.degree
    Y0 = to_dev(workloads.complex_normal(w.seed + 100, (N, nv)))
    X = torch.empty_like(Y0)
    lam = R.rcf_rayleigh_ritz(g.ctx, g.op, Y0, X)
    lo, hi = R.rcf_lanczos_bounds(g.ctx, g.op, w.lanczos, to_dev(workloads.complex_normal(w.seed + 200, N))[0])
    bounds = (float(lam.min()), float(lam.max()), hi)
    V = torch.from_numpy(g.V).cuda()
    B = torch.from_numpy(g.B).cuda()
    h = torch.from_numpy(np.ascontiguousarray(g.params["proj_h"])).cuda()

    def loss(Vt, Bt, ht, G, nlow=32):
        Y = RChFSIFilter.apply(Vt, Bt, ht, opw, X, lam, bounds, q, R.RCF_FP64, w.ckpt)
        th = RitzValues.apply(Y, Vt, Bt, ht, opw)
        return th[:nlow].sum() + torch.vdot(G.reshape(-1), Y.reshape(-1)).real

    with torch.no_grad():
        Yq = RChFSIFilter.apply(V, B, h, opw, X, lam, bounds, q, R.RCF_FP64, w.ckpt)
    G = to_dev(workloads.complex_normal(w.seed + 300, (N, nv)))
    G = G / torch.linalg.norm(G) / torch.linalg.norm(Yq) * 10.0

    Vr, Br, hr = V.clone().requires_grad_(), B.clone().requires_grad_(), h.clone().requires_grad_()
    L = loss(Vr, Br, hr, G)
    L.backward()
    gV, gB, gh = Vr.grad.cpu().numpy(), Br.grad.cpu().numpy(), hr.grad.cpu().numpy()

    rng = np.random.default_rng(w.seed)
    entries = ([("V", (int(rng.integers(V.shape[0])), int(rng.integers(V.shape[1])))) for _ in range(120)]
               + [("B", (int(rng.integers(3)), int(rng.integers(V.shape[0])), int(rng.integers(V.shape[1]))))
                  for _ in range(72)]
               + [("h", (a, j)) for a in range(w.natoms) for j in range(2)])
    assert len(entries) == 200
    step = 1e-5
    fd, an = [], []
    with torch.no_grad():
        for kind, idx in entries:
            vals = []
            for sgn in (1.0, -1.0):
                Vp, Bp, hp = V.clone(), B.clone(), h.clone()
                t = {"V": Vp, "B": Bp, "h": hp}[kind]
                t[idx] += sgn * step
                vals.append(float(loss(Vp, Bp, hp, G)))
            fd.append((vals[0] - vals[1]) / (2 * step))
            an.append({"V": gV, "B": gB, "h": gh}[kind][idx])
    fd, an = np.array(fd), np.array(an)
    err = np.linalg.norm(fd - an) / np.linalg.norm(fd)
    g.close()
    assert err < 1e-6, err


def test_ritz_cotangent_matches_oracle(small):
    """rcf_ritz_cotangent against the oracle's Ritz-value loss head: for L = sum of the lowest
    nlow Ritz values of span(Y) (+ Re <G, Y>, added on the host since it is linear in Y), the
    cotangent Ybar and the direct derivative sum_j x_j^H dH x_j in V, B and the couplings."""
    import torch
    from oracle import ritz_loss_head
    from paper_2605_30128_gb300 import rchfsi as R
    H = small.H
    nv, nlow = 6, 4
    Y = workloads.complex_normal(43, (H.N, nv))
    G = np.zeros_like(Y)
    _, oYbar, (gV, gB, gh) = ritz_loss_head(H, Y, G, nlow)
    oV = H.node_to_quadrature(gV)
    oB = np.stack([H.node_to_quadrature(gB[d]) for d in range(3)])
    Yd = to_dev(Y)
    Xr = torch.empty_like(Yd)
    theta = R.rcf_rayleigh_ritz(small.g.ctx, small.g.op, Yd.clone(), Xr)
    tb = np.zeros(nv)
    tb[:nlow] = 1.0
    Ybar = torch.empty_like(Yd)
    dV = torch.zeros(small.V.shape, dtype=torch.float64, device="cuda")
    dB = torch.zeros(small.B.shape, dtype=torch.float64, device="cuda")
    dh = np.zeros((2, 2))
    for _ in range(2):                       # the derivative parts accumulate; Ybar is overwritten
        R.rcf_ritz_cotangent(small.g.ctx, small.g.op, Yd, Xr, theta, tb, Ybar, dV, dB, dh)
    assert rel(to_host(Ybar), oYbar) < 1e-10
    assert np.abs(to_host(Ybar) - oYbar).max() < 1e-10 * np.abs(oYbar).max()
    assert rel(dV.cpu().numpy() / 2, oV) < 1e-10
    assert rel(dB.cpu().numpy() / 2, oB) < 1e-10
    assert rel(dh / 2, gh) < 1e-10
