"""Timing of the tall products of Rayleigh-Ritz and of the Poisson solve through the C ABI.

    python -m paper_2605_30128_gb300.products --rows 3456000 --cols 1024
    python -m paper_2605_30128_gb300.products --poisson --ncell 20 --p 5
    python -m paper_2605_30128_gb300.products --fullmass --ncell 20 --p 5 --nvec 64

Tall products (Algorithm 1, RR step; Section III-C-4): C = Y^H Y (rcf_inner) and X = Y Q
(rcf_rotate) for a seeded complex block Y of `rows` complex rows and `cols` columns, in each
requested arithmetic (tc: FP64-accurate on the bf16 tensor cores; mixed: the rotation with its
off-diagonal part at FP32 level; fp64: cuBLAS), CUDA events on the library's stream, best of
`--reps`.  The JSON line gives the times, the bf16 tensor work per second of the tc calls
(28 digit products of 2 m n K flops) and, for fp64, the FP64 rate.

Full mass (Section III-A; Section III-B-2): one FP32 R-ChFSI step H D^-1 with the consistent
mass and the Gauss-point potential, one M X, and the lumped step on the same mesh.

Poisson (Section III-B-1; Algorithm pcg_fusion): K x on the scalar nodal field of a periodic
ncell^3 mesh of degree p (cell edge 2 bohr) and one PCG solve with a degree-5
Chebyshev-Jacobi preconditioner to an absolute residual of 1e-10.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

from . import rchfsi as R


def _timer(torch, stream):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best
    return timed


def products(rows: int, cols: int, ariths, reps: int) -> dict:
    import torch
    stream = torch.cuda.current_stream()
    timed = _timer(torch, stream)
    ctx = R.rcf_create(0, stream)
    try:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(1)
        Y = torch.randn((cols, rows), dtype=torch.complex128, device="cuda", generator=gen) / rows ** 0.5
        Q = torch.randn((cols, cols), dtype=torch.complex128, device="cuda", generator=gen) / cols ** 0.5
        C = torch.zeros((cols, cols), dtype=torch.complex128, device="cuda")
        X = torch.empty_like(Y)
        out = {"rows": rows, "cols": cols}
        codes = {"tc": R.RCF_RR_TC, "mixed": R.RCF_RR_MIXED, "fp64": R.RCF_RR_FP64}
        tc_flops = 28 * 2.0 * cols * (2 * cols) * (2 * rows)
        for a in ariths:
            code = codes[a]
            if a != "mixed":
                ms = timed(lambda: R.rcf_inner(ctx, Y, Y, C, None, code), reps)
                out[f"inner_{a}_ms"] = ms
            ms_r = timed(lambda: R.rcf_rotate(ctx, Y, Q, X, code), reps)
            out[f"rotate_{a}_ms"] = ms_r
            if a == "tc":
                out["inner_tc_bf16_tflops"] = tc_flops / (out["inner_tc_ms"] * 1e-3) / 1e12
                out["rotate_tc_bf16_tflops"] = tc_flops / (ms_r * 1e-3) / 1e12
            if a == "fp64":
                out["inner_fp64_tflops"] = 8.0 * cols * cols * rows / (out["inner_fp64_ms"] * 1e-3) / 1e12
                out["rotate_fp64_tflops"] = 8.0 * cols * cols * rows / (ms_r * 1e-3) / 1e12
        return out
    finally:
        R.rcf_destroy(ctx)


def poisson(ncell: int, p: int, reps: int) -> dict:
    import torch
    stream = torch.cuda.current_stream()
    timed = _timer(torch, stream)
    ctx = R.rcf_create(0, stream)
    mesh = R.rcf_mesh_create(ctx, ncell, 2.0 * ncell, p)
    try:
        n = R.rcf_mesh_info(mesh)[0]
        gen = torch.Generator(device="cuda")
        gen.manual_seed(2)
        x = torch.randn((n,), dtype=torch.float64, device="cuda", generator=gen)
        y = torch.empty_like(x)
        kx = timed(lambda: R.rcf_laplacian(ctx, mesh, x, y), reps)
        f = torch.randn((n,), dtype=torch.float64, device="cuda", generator=gen)
        f -= f.mean()
        xs = torch.zeros_like(f)
        t0 = time.perf_counter()
        it, res = R.rcf_poisson_pcg(ctx, mesh, f, xs, 5, 0.0, 0.0, 1e-10, 5000)
        torch.cuda.synchronize()
        return {"ncell": ncell, "p": p, "nodes": n, "kx_ms": kx, "kx_dofs_per_s": n / (kx * 1e-3),
                "pcg_iterations": it, "pcg_residual": res, "pcg_ms": (time.perf_counter() - t0) * 1e3}
    finally:
        R.rcf_mesh_destroy(mesh)
        R.rcf_destroy(ctx)


def fullmass(ncell: int, p: int, nvec: int, reps: int) -> dict:
    """One FP32 R-ChFSI step (H D^-1) with the full consistent mass (n_q = p + 2) and one M X on
    a periodic ncell^3 mesh of degree p (cell edge 2 bohr, a seeded Gaussian-sum potential and a
    smooth magnetic field at the Gauss points, no projectors), beside the lumped step."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    timed = _timer(torch, stream)
    ctx = R.rcf_create(0, stream)
    mesh = R.rcf_mesh_create(ctx, ncell, 2.0 * ncell, p)
    ops = []
    try:
        n, ncells, _ = R.rcf_mesh_info(mesh)
        nq = p + 2
        op = R.rcf_op_create(ctx, mesh)
        ops.append(op)
        R.rcf_op_set_gauss(ctx, op, nq)
        xq = R.rcf_op_gauss_points(ctx, op, ncells, nq).reshape(-1, 3)
        L = 2.0 * ncell
        V = -2.0 * np.exp(-((xq - L / 2) ** 2).sum(axis=1) / 8.0)
        B = 0.05 * np.stack([np.cos(2 * np.pi * xq[:, 0] / L), np.sin(2 * np.pi * xq[:, 1] / L),
                             np.cos(2 * np.pi * xq[:, 2] / L)])
        R.rcf_potential_set(ctx, op, V.reshape(ncells, -1), B.reshape(3, ncells, -1))
        lumped = R.rcf_op_create(ctx, mesh)
        ops.append(lumped)
        R.rcf_potential_set(ctx, lumped, np.zeros((ncells, (p + 1) ** 3)), None)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(3)
        N = 2 * n
        Zk, Zm, Rr = (torch.randn((nvec, N), dtype=torch.complex64, device="cuda", generator=gen) for _ in range(3))
        O = torch.empty_like(Zk)
        g = torch.full((nvec,), 0.25, dtype=torch.float64, device="cuda")
        st = lambda o: R.rcf_cheb_step(ctx, o, R.RCF_FORM_H_DINV, R.RCF_FP32, Zk, Zm, Rr, 0.1, -0.5, -1.0, g, O)
        fm_ms = timed(lambda: st(op), reps)
        lumped_ms = timed(lambda: st(lumped), reps)
        m_ms = timed(lambda: R.rcf_mass_apply(ctx, op, Zk, O, R.RCF_FP32), reps)
        return {"ncell": ncell, "p": p, "gauss_points": nq, "vectors": nvec, "step_ms": fm_ms,
                "lumped_step_ms": lumped_ms, "mass_apply_ms": m_ms,
                "step_gbs_at_32_bytes_per_unit": 32.0 * N * nvec / (fm_ms * 1e-3) / 1e9}
    finally:
        for o in ops:
            R.rcf_op_destroy(o)
        R.rcf_mesh_destroy(mesh)
        R.rcf_destroy(ctx)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=262144)
    ap.add_argument("--cols", type=int, default=256)
    ap.add_argument("--arith", default="tc,mixed,fp64")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--poisson", action="store_true")
    ap.add_argument("--fullmass", action="store_true")
    ap.add_argument("--nvec", type=int, default=64)
    ap.add_argument("--ncell", type=int, default=20)
    ap.add_argument("--p", type=int, default=5)
    a = ap.parse_args(argv)
    from .build import build
    build()
    if a.poisson:
        print(json.dumps(poisson(a.ncell, a.p, a.reps)))
    elif a.fullmass:
        print(json.dumps(fullmass(a.ncell, a.p, a.nvec, a.reps)))
    else:
        print(json.dumps(products(a.rows, a.cols, [s for s in a.arith.split(",") if s], a.reps)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
