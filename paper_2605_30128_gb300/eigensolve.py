"""Algorithm 1 (R-ChFSI / ChFSI subspace iteration) on one GPU through the C ABI, with each
phase timed on the stream: residual check, filter, Cholesky-QR2, Rayleigh-Ritz.

    python -m paper_2605_30128_gb300.eigensolve --workload cfg5 --cycles 2
    python -m paper_2605_30128_gb300.eigensolve --workload cfg3 --nvec 256 --block 256 \\
        --cycles 30 --tol 1e-8 --nwanted 224
    python -m paper_2605_30128_gb300.eigensolve --workload cfg4 --gauss 6 --cycles 40 \\
        --runs rchfsi_fp64,rchfsi_fp32,chfsi_fp64      # full consistent mass, diagonal D

Every run starts from the same seeded block and the same initial Rayleigh-Ritz step, then
runs each requested filter (default: mixed R-ChFSI with the double-float residual, mixed
R-ChFSI with the FP64 residual, FP64 ChFSI) for the given number of cycles or until the
largest residual norm of the wanted vectors, ||H x_j - theta_j M x_j||, falls below tol.
The JSON line reports per cycle and phase times and, for every run after the last FP64 one,
the largest difference of its wanted Ritz values from that FP64 run.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

import workloads

from . import rchfsi as R
from .problem import GPUProblem

RUNS = {
    "rchfsi_fp32_df": (R.RCF_RCHFSI, R.RCF_FP32_DF),
    "rchfsi_fp32": (R.RCF_RCHFSI, R.RCF_FP32),
    "rchfsi_fp64": (R.RCF_RCHFSI, R.RCF_FP64),
    "chfsi_fp64": (R.RCF_CHFSI, R.RCF_FP64),
}


class Timer:
    """Elapsed milliseconds of a call on the stream, bracketed by CUDA events."""

    def __init__(self, torch, stream):
        self.t, self.s = torch, stream
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def __call__(self, fn):
        self.e0.record(self.s)
        out = fn()
        self.e1.record(self.s)
        self.t.cuda.synchronize()
        return out, self.e0.elapsed_time(self.e1)


def use_full_mass(prob, w, nq):
    """Switch the problem's operator to the full consistent mass with nq Gauss points per
    direction (Section III-A; Section III-B-2): the same synthetic V, B and projectors,
    V and B evaluated at the Gauss points."""
    ctx, op = prob.ctx, prob.op
    R.rcf_op_set_gauss(ctx, op, nq)
    xq = R.rcf_op_gauss_points(ctx, op, prob.ncells, nq).reshape(-1, 3)
    prm = prob.params
    V = workloads.gaussian_sum_potential(xq, prm["centres"], prm["depths"], prm["widths"], prm["L"])
    B = workloads.smooth_periodic_field(xq, prm["kvec"], prm["amps"], prm["phases"], prm["L"], prm["bmax"])
    R.rcf_potential_set(ctx, op, V.reshape(prob.ncells, -1), B.reshape(3, prob.ncells, -1))
    if w.natoms > 0:
        R.rcf_projectors_set(ctx, op, prm["atoms"], prm["proj_width"], prm["proj_h"])


def run(w, runs, cycles, tol, nwanted, seed=0, device=0, rr_arith=None, gauss=0):
    import torch
    dev = torch.device("cuda", device)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    tm = Timer(torch, stream)
    prob = GPUProblem(w, device=device, stream=stream)
    if gauss:
        use_full_mass(prob, w, gauss)
    ctx, op = prob.ctx, prob.op
    if rr_arith is not None:
        R.rcf_set_rr_arith(ctx, rr_arith)
    N, nvec = prob.N, w.nvec
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed + 100 + seed)
    X0 = torch.randn((nvec, N), dtype=torch.complex128, device=dev, generator=gen)
    v0 = torch.randn((N,), dtype=torch.complex128, device=dev, generator=gen)
    (lo, lmax), t_lz = tm(lambda: R.rcf_lanczos_bounds(ctx, op, w.lanczos, v0))
    del v0
    Y = torch.empty_like(X0)
    # initial Rayleigh-Ritz on the start block, shared by all runs
    _, t_q0 = tm(lambda: R.rcf_cholqr2(ctx, op, X0))
    Xinit = torch.empty_like(X0)
    lam0, t_r0 = tm(lambda: R.rcf_rayleigh_ritz_orth(ctx, op, X0, Xinit))
    del X0
    X = torch.empty_like(Xinit)
    cn = torch.zeros(nvec, dtype=torch.float64, device=dev)
    out = {"workload": f"{w.name}: {w.ncell}^3 cells, p={w.p}, {N:,} complex DoF, {w.natoms} atoms, "
                       f"{nvec} vectors in blocks of {w.block}, degree {w.degree}"
                       + (f", full consistent mass with {gauss}^3 Gauss points per cell" if gauss else ""),
           "lanczos_ms": t_lz, "initial_cholqr2_ms": t_q0, "initial_rr_ms": t_r0,
           "lambda_max": lmax, "nwanted": nwanted, "tol": tol, "runs": {}}
    ref_name, ref_lam = None, None
    for name in runs:
        mode, prec = RUNS[name]
        X.copy_(Xinit)
        lam = lam0.copy()
        hist = []
        def residual_norms():
            # column norms of H X - M X Lambda, one band block at a time (bounded scratch)
            for b0 in range(0, nvec, w.block):
                b1 = min(nvec, b0 + w.block)
                R.rcf_residual(ctx, op, X[b0:b1], lam[b0:b1], None, cn[b0:b1])

        for c in range(cycles):
            _, t_res = tm(residual_norms)
            res = cn.cpu().numpy()
            rmax = float(res[:nwanted].max())
            if rmax < tol:
                hist.append({"cycle": c, "max_residual": rmax, "residual_ms": t_res})
                break
            bounds = (float(lam.min()), float(lam.max()), lmax)
            _, t_f = tm(lambda: R.rcf_filter(ctx, op, X, lam, w.degree, bounds, mode, prec, w.block, Y))
            _, t_q = tm(lambda: R.rcf_cholqr2(ctx, op, Y))
            lam, t_r = tm(lambda: R.rcf_rayleigh_ritz_orth(ctx, op, Y, X))
            hist.append({"cycle": c, "max_residual": rmax, "residual_ms": t_res, "filter_ms": t_f,
                         "cholqr2_ms": t_q, "rayleigh_ritz_ms": t_r})
        full = [h for h in hist if "filter_ms" in h]
        rec = {"cycles": len(full), "final_max_residual": hist[-1]["max_residual"], "history": hist,
               "ritz_wanted_min_max": [float(lam[0]), float(lam[nwanted - 1])]}
        if full:
            for k in ("filter_ms", "cholqr2_ms", "rayleigh_ritz_ms", "residual_ms"):
                rec["mean_" + k] = float(np.mean([h[k] for h in full]))
            per = rec["mean_filter_ms"] + rec["mean_cholqr2_ms"] + rec["mean_rayleigh_ritz_ms"]
            rec["cycle_ms"] = per + rec["mean_residual_ms"]
            rec["split"] = {"filter": rec["mean_filter_ms"] / per, "cholqr2": rec["mean_cholqr2_ms"] / per,
                            "rayleigh_ritz": rec["mean_rayleigh_ritz_ms"] / per}
        if prec == R.RCF_FP64:
            ref_name, ref_lam = name, lam.copy()
        elif ref_lam is not None:
            rec["max_ritz_diff_vs_" + ref_name] = float(np.max(np.abs(lam[:nwanted] - ref_lam[:nwanted])))
        rec["_lam"] = lam
        out["runs"][name] = rec
    # runs before the first FP64 run are compared once it exists
    for name, rec in out["runs"].items():
        if ref_lam is not None and "max_ritz_diff_vs_" + str(ref_name) not in rec and name != ref_name:
            rec["max_ritz_diff_vs_" + ref_name] = float(np.max(np.abs(rec["_lam"][:nwanted] - ref_lam[:nwanted])))
    for rec in out["runs"].values():
        rec.pop("_lam")
    prob.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="cfg5")
    ap.add_argument("--nvec", type=int, default=None)
    ap.add_argument("--block", type=int, default=None)
    ap.add_argument("--degree", type=int, default=None)
    ap.add_argument("--cycles", type=int, default=5)
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--nwanted", type=int, default=None,
                    help="wanted vectors (default: all but a buffer of max(4, nvec/10))")
    ap.add_argument("--runs", default="rchfsi_fp32_df,rchfsi_fp32,chfsi_fp64")
    ap.add_argument("--gauss", type=int, default=0,
                    help="full consistent mass with this many Gauss points per direction (0: lumped)")
    ap.add_argument("--rr", default="tc", choices=["fp64", "df", "tc", "mixed"],
                    help="tall products of Cholesky-QR2 and Rayleigh-Ritz: cuBLAS FP64, double-float, tensor "
                         "cores, or tensor cores with the mixed-precision rotation")
    a = ap.parse_args(argv)
    over = {k: v for k, v in (("nvec", a.nvec), ("block", a.block), ("degree", a.degree)) if v}
    w = workloads.workload(a.workload, **over)
    nw = a.nwanted or w.nvec - max(4, w.nvec // 10)
    runs = [r for r in a.runs.split(",") if r]
    for r in runs:
        if r not in RUNS:
            raise SystemExit(f"unknown run {r}; choose from {', '.join(RUNS)}")
    # FP64 runs first so the others can be compared as they finish
    runs.sort(key=lambda r: RUNS[r][1] != R.RCF_FP64)
    t0 = time.time()
    out = run(w, runs, a.cycles, a.tol, nw,
              rr_arith={"fp64": R.RCF_RR_FP64, "df": R.RCF_RR_DF, "tc": R.RCF_RR_TC,
                        "mixed": R.RCF_RR_MIXED}[a.rr], gauss=a.gauss)
    out["rr_arith"] = a.rr
    out["wall_s"] = time.time() - t0
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
