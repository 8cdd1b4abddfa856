#!/usr/bin/env python
"""Throughput of the mixed-precision R-ChFSI filter on one GB300, in filtered DoF*vec*deg/s.

Workload (default): periodic 20^3 cells, p = 5 (100^3 nodes, 2,000,000 complex
spinor DoF), 32 atoms with spin-orbit projectors, 1024 spinor vectors filtered
in band blocks of 256 at degree 40.  The recurrence runs in complex64 (FP32
stencil products); X, the residual R = HX - MX Lambda and the recovery are
complex128 (RCF_FP32: the paper's split, R in FP64).  A step is one rcf_filter
call over all 1024 vectors: X -> Y_q including the residual and the recovery.
Units per step = 2M * nvec * degree.  The same filter with R evaluated in
double-float arithmetic (RCF_FP32_DF) and with 16-bit storage is reported
beside it.

Also reported on the same JSON line: the dominant kernel (the FP32 recurrence
step) against the measured HBM copy bandwidth, the FP64 ChFSI filter on the
same mesh and block, an end-to-end figure through the C ABI with host
buffers, the CPU oracle on a bounded sample, sampled SM clocks, and the
number of this library's kernel launches in the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank filters its own band of 1024
vectors (band partitioning with one GPU per column group: the filter needs no
communication), so per-GPU work is fixed ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filtered DoF·vec·deg/s: mixed-prec R-ChFSI vs FP64 ChFSI at ≤1e-7 Ha eig err"
UNIT = "DoF·vec·deg/s"
BYTES_PER_UNIT = 32.0   # read Z_k, Z_{k-1}, R (complex64) + write Z_{k+1}
BYTES_PER_UNIT_BFP12 = 27.0   # as above with R read from its 12-bit BFP stream (3 B per DoF)
KERNEL_SRC = os.path.join(ROOT, "paper_2605_30128_gb300", "csrc", "stencil.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg3")
    ap.add_argument("--nvec", type=int, default=None, help="override (profiling runs only)")
    ap.add_argument("--block", type=int, default=None)
    ap.add_argument("--degree", type=int, default=None)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64, e2e and CPU legs (profiling runs only)")
    ap.add_argument("--codec-only", action="store_true",
                    help="time only the block floating-point codec on one residual block (prints its object)")
    return ap.parse_args()


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workloads_mod():
    import workloads
    return workloads


def workload_of(args):
    import workloads
    over = {}
    if args.nvec:
        over["nvec"] = args.nvec
    if args.block:
        over["block"] = args.block
    if args.degree:
        over["degree"] = args.degree
    return workloads.workload(args.workload, **over)


def describe(w) -> str:
    return (f"{w.name}: periodic {w.ncell}^3 cells, p={w.p}, side {w.side:g} bohr, "
            f"{w.ndof:,} complex spinor DoF, {w.natoms} spin-orbit atoms, {w.nvec} vectors "
            f"in blocks of {w.block}, degree {w.degree}")


# ----------------------------------------------------------------------------------------
# CPU oracle on a bounded sample (the reference arm and the cpu_baseline leg)
# ----------------------------------------------------------------------------------------

def oracle_setup(w):
    import numpy as np
    import workloads
    from oracle import Hamiltonian, Mesh
    prm = workloads.draw_parameters(w)
    m = Mesh(w.ncell, w.side, w.p)
    q = m.quad_coords().reshape(-1, 3)
    V = workloads.gaussian_sum_potential(q, prm["centres"], prm["depths"], prm["widths"], prm["L"])
    B = workloads.smooth_periodic_field(q, prm["kvec"], prm["amps"], prm["phases"], prm["L"], prm["bmax"])
    H = Hamiltonian(m, V.reshape(m.ncells, m.nloc), B.reshape(3, m.ncells, m.nloc), prm["atoms"],
                    prm["proj_width"], prm["proj_h"])
    return H


def oracle_sample(H, nv: int, q: int, seed: int):
    """Time the oracle's R-ChFSI filter (FP64, scipy sparse) on nv vectors at degree q."""
    import numpy as np
    import workloads
    from oracle import rchfsi_filter
    X = workloads.complex_normal(seed, (H.N, nv))
    lam = np.linspace(-1.0, 0.5, nv)
    t0 = time.perf_counter()
    rchfsi_filter(H, X, lam, -1.5, 1.0, 60.0, q)
    dt = time.perf_counter() - t0
    return H.N * nv * q / dt, dt


ORACLE_NV, ORACLE_Q = 16, 6


def run_reference(args):
    ws, rank, local = dist_init(args)
    if rank != 0:
        return 0
    w = workload_of(args)
    H = oracle_setup(w)
    for i in range(args.warmup):
        oracle_sample(H, ORACLE_NV, ORACLE_Q, 500 + i)
    times, vals = [], []
    for i in range(args.steps):
        v, dt = oracle_sample(H, ORACLE_NV, ORACLE_Q, 600 + i)
        vals.append(v)
        times.append(dt)
    value = statistics.median(vals)
    sample = (f"oracle R-ChFSI filter (NumPy/SciPy FP64, CSR sparse H) on the full {w.ncell}^3 p={w.p} mesh, "
              f"{ORACLE_NV} vectors, degree {ORACLE_Q} per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": describe(w)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host_cores": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------

def traffic_record():
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None when
    the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
        return rec if rec.get("kernel_sha256") == h else None
    except Exception:
        return None



def measured_hbm_peak():
    """(GB/s, source): the HBM copy bandwidth measured on this GPU model ("measured"), else the
    fallback figure of an earlier GB300 measurement ("fallback")."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


HEADLINE_PRECISION = ("recurrence and stencil products complex64 (FP32); X, the residual R = HX - MX Lambda "
                      "and the recovery complex128 (FP64), R rounded to complex64 for the recurrence "
                      "(RCF_FP32: the paper's split)")


def assemble_line(w, ws: int, steps: int, warmup: int, m: dict) -> dict:
    """The bench's JSON line from the measurements in m (times in ms, per rank maxima).

    Keys of m: ms (headline step), launches, clocks, N, nvec, degree, l2_gb, peak (GB/s, source),
    traffic (record or None), variants_ms {df_residual, fp16_storage, bf16_storage}, kernel
    {blk, k_ms, step_ms, k16_ms}, residual {df_ms, fp64_ms}; optional fp64_chfsi {blk, f64_ms,
    mix_ms}, e2e {ms, ne, h2d, d2h, sample, link}, adjoint, bfp_codec, cpu_baseline {value, dt}."""
    N, nvec, q = m["N"], m["nvec"], m["degree"]
    units = float(N) * nvec * q
    rate = lambda ms: units * ws / (ms * 1e-3)
    peak, peak_source = m["peak"]
    line = {
        "metric": METRIC, "value": rate(m["ms"]), "unit": UNIT, "n_gpus": ws, "steps": steps,
        "warmup": warmup, "ms_per_step": m["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe(w), "precision": HEADLINE_PRECISION,
                   "l2": "inputs larger than L2 (X and Y are %.1f GB each)" % m["l2_gb"],
                   "parallelism": "band partitioning, one GPU per column group (no filter communication)"
                                  if ws > 1 else "single GPU"},
        "gpu_launches": int(m["launches"]),
        "clocks": m["clocks"],
    }
    vm = m["variants_ms"]
    line["variants"] = {
        "df_residual": {"value": rate(vm["df_residual"]), "unit": UNIT, "ms_per_step": vm["df_residual"],
                        "precision": "as the headline with R evaluated in double-float arithmetic (pairs of "
                                     "FP32, about 2^-46 of the term magnitudes; RCF_FP32_DF)"},
        "fp16_storage": {"value": rate(vm["fp16_storage"]), "unit": UNIT, "ms_per_step": vm["fp16_storage"],
                         "precision": "Z_k, Z_{k-1}, R stored as binary16 pairs (R scaled per column), "
                                      "products in FP32, double-float residual (RCF_FP16)"},
        "bf16_storage": {"value": rate(vm["bf16_storage"]), "unit": UNIT, "ms_per_step": vm["bf16_storage"],
                         "precision": "as fp16_storage with bfloat16 (RCF_BF16)"},
    }
    if "bfp12_residual" in vm:
        line["variants"]["bfp12_residual"] = {
            "value": rate(vm["bfp12_residual"]), "unit": UNIT, "ms_per_step": vm["bfp12_residual"],
            "precision": "as the headline with R (FP64, rounded to FP32) kept as a 12-bit block floating-point "
                         "stream read by every step (RCF_FP32_BFP12)"}
    k = m["kernel"]
    blk = k["blk"]
    alg = BYTES_PER_UNIT * N * blk
    achieved = alg / (k["k_ms"] * 1e-3) / 1e9
    tr = m["traffic"]
    line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": (tr["bytes_per_launch_full_block"] if tr else None),
                        "kernel": "step_kernel<float,%d> (FP32 R-ChFSI recurrence step, %d vectors)" % (w.p, blk),
                        "kernel_ms": k["k_ms"], "algorithmic_bytes": alg, "peak_source": peak_source,
                        "step_with_projectors_ms": k["step_ms"]}
    a16 = 16.0 * N * blk / (k["k16_ms"] * 1e-3) / 1e9
    line["roofline_fp16_step"] = {"bound": "hbm", "achieved": a16, "peak": peak, "unit": "GB/s",
                                  "frac": a16 / peak, "kernel_ms": k["k16_ms"], "algorithmic_bytes": 16.0 * N * blk,
                                  "kernel": "step_kernel<float,__half,%d> (recurrence step, vectors stored as "
                                            "binary16)" % w.p}
    if "kbfp_ms" in k:
        ab = BYTES_PER_UNIT_BFP12 * N * blk
        abfp = ab / (k["kbfp_ms"] * 1e-3) / 1e9
        line["roofline_bfp12_step"] = {"bound": "hbm", "achieved": abfp, "peak": peak, "unit": "GB/s",
                                       "frac": abfp / peak, "kernel_ms": k["kbfp_ms"], "algorithmic_bytes": ab,
                                       "kernel": "step_kernel<float,%d> reading R from a 12-bit BFP stream "
                                                 "(27 B per unit)" % w.p}
    r = m["residual"]
    line["residual"] = {"fp64_ms": r["fp64_ms"], "double_float_ms": r["df_ms"], "vectors": blk,
                        "note": "R = H X - M X Lambda of one block, spin-orbit terms included"}
    if "fp64_chfsi" in m:
        f = m["fp64_chfsi"]
        line["fp64_chfsi"] = {"value": float(N) * f["blk"] * q * ws / (f["f64_ms"] * 1e-3), "unit": UNIT,
                              "ms_one_block": f["f64_ms"], "mixed_rchfsi_ms_one_block": f["mix_ms"],
                              "speedup_mixed_over_fp64": f["f64_ms"] / f["mix_ms"],
                              "sample": "one block of %d vectors, degree %d; mixed = the headline "
                                        "arithmetic (RCF_FP32)" % (f["blk"], q)}
    if "e2e" in m:
        e = m["e2e"]
        line["e2e"] = {"value": float(N) * e["ne"] * q * ws / (e["ms"] * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": int(e["h2d"]), "d2h_bytes_per_step": int(e["d2h"]),
                       "ms_per_step": e["ms"], "sample": e["sample"], "link": e["link"],
                       "calls_ms": e.get("calls_ms"),
                       "call": "rcf_filter_host, RCF_FP32 (pinned host X and Y; wall clock around the "
                               "synchronising call)"}
    for key in ("adjoint", "bfp_codec", "poisson", "fullmass"):
        if key in m:
            line[key] = m[key]
    if "cpu_baseline" in m:
        c = m["cpu_baseline"]
        line["cpu_baseline"] = {"value": c["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"oracle R-ChFSI filter (NumPy/SciPy FP64, single-threaded CSR "
                                          f"products) on the full mesh, {ORACLE_NV} vectors, degree "
                                          f"{ORACLE_Q}: {c['dt']:.1f} s",
                                "host_cores": os.cpu_count()}
    return line


def codec_leg(R, ctx, op, Xb, ritz_b, peak, stream):
    """The block floating-point codec (Section III-C-3) on the double-float residual of one
    block Xb (256 vectors of the 20^3 p = 5 workload: 1.02e9 FP32 values, 4.1 GB > L2):
    encode and decode at each rate, 5 launches each timed with CUDA events on the library's
    stream; algorithmic bytes = 4 per value + the stream.  Any failure is reported in the
    returned object (the codec is reported beside the filter, never instead of it)."""
    import torch
    try:
        Rh = torch.empty(Xb.shape, dtype=torch.complex64, device=Xb.device)
        R.rcf_residual_df(ctx, op, Xb, ritz_b, Rh)
        rv = Rh.view(torch.float32).reshape(-1)
        n_r = rv.numel()
        dec = torch.empty_like(rv)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out = {}
        for nbits in R.RCF_BFP_RATES:
            sbuf = torch.empty(R.rcf_bfp_stream_bytes(n_r, nbits), dtype=torch.uint8, device=Xb.device)
            R.rcf_bfp_encode(ctx, rv, nbits, sbuf)
            R.rcf_bfp_decode(ctx, sbuf, nbits, dec)
            torch.cuda.synchronize()
            reps = 5
            ev0.record(stream)
            for _ in range(reps):
                R.rcf_bfp_encode(ctx, rv, nbits, sbuf)
            ev1.record(stream)
            torch.cuda.synchronize()
            e_ms = ev0.elapsed_time(ev1) / reps
            ev0.record(stream)
            for _ in range(reps):
                R.rcf_bfp_decode(ctx, sbuf, nbits, dec)
            ev1.record(stream)
            torch.cuda.synchronize()
            d_ms = ev0.elapsed_time(ev1) / reps
            moved = 4.0 * n_r + sbuf.numel()
            num = den = 0.0
            for c0 in range(0, n_r, 1 << 27):
                a = rv[c0:c0 + (1 << 27)].double()
                num += float(((dec[c0:c0 + (1 << 27)].double() - a) ** 2).sum())
                den += float((a * a).sum())
            out[str(nbits)] = {
                "encode_ms": e_ms, "decode_ms": d_ms,
                "encode_gbs": moved / (e_ms * 1e6), "decode_gbs": moved / (d_ms * 1e6),
                "encode_frac": moved / (e_ms * 1e6) / peak, "decode_frac": moved / (d_ms * 1e6) / peak,
                "stream_bytes": int(sbuf.numel()), "rel_error_fro": (num / den) ** 0.5}
            del sbuf
        return dict(out, values=n_r, peak_gbs=peak, bound="hbm",
                    data="double-float residual R of one %d-vector block, as FP32" % Xb.shape[0],
                    note="algorithmic bytes = 4 per value + the stream; frac of the measured copy bandwidth")
    except Exception as exc:
        return {"error": repr(exc)[:300]}

def poisson_leg(R, ctx, mesh, w, dev, gen, timed):
    """K x on the scalar nodal field of the mesh (10 launches timed) and one PCG solve with a
    degree-5 Chebyshev-Jacobi preconditioner (interval from the Gershgorin bound) of a seeded
    zero-sum right-hand side to an absolute residual of 1e-10 (the paper's setting, p = 7 there).
    Any failure is reported in the returned object."""
    import torch
    try:
        n = w.nnodes
        x = torch.randn((n,), dtype=torch.float64, device=dev, generator=gen)
        y = torch.empty_like(x)
        R.rcf_laplacian(ctx, mesh, x, y)
        kx_ms = timed(lambda: R.rcf_laplacian(ctx, mesh, x, y), 10)
        f = torch.randn((n,), dtype=torch.float64, device=dev, generator=gen)
        f -= f.mean()
        xs = torch.zeros_like(f)
        t0 = time.perf_counter()
        it, res = R.rcf_poisson_pcg(ctx, mesh, f, xs, 5, 0.0, 0.0, 1e-10, 5000)
        torch.cuda.synchronize()
        pcg_ms = (time.perf_counter() - t0) * 1e3
        p = w.p
        taps = 3.0 * (2 * p + 1 + (p - 1) * (p + 1)) / p        # stencil taps per node, 3 directions
        flops = 2.0 * taps + 9.0                                   # FMA per tap; weights and sums
        return {"nodes": n, "kx_ms": kx_ms, "kx_dofs_per_s": n / (kx_ms * 1e-3),
                "kx_fp64_tflops": n * flops / (kx_ms * 1e-3) / 1e12, "flop_per_dof": flops,
                "fp64_peak_tflops_nominal": 1.25, "kx_frac_of_nominal_fp64": n * flops / (kx_ms * 1e-3) / 1.25e12,
                "pcg_iterations": it, "pcg_residual": res, "pcg_ms": pcg_ms,
                "pcg_ms_per_iteration": pcg_ms / max(it, 1), "chebyshev_degree": 5,
                "note": "scalar periodic FE Laplacian on the bench mesh, FP64; PCG wall clock includes one "
                        "host read of the residual norm per iteration"}
    except Exception as exc:
        return {"error": repr(exc)[:300]}


def fullmass_leg(R, ctx, prob, w, dev, gen, timed, nvec=64):
    """One FP32 R-ChFSI step (Eq. rChFSIrecurrence, H D^-1 with the full consistent mass,
    n_q = p + 2 Gauss points per direction, the Gauss-point potential and the projectors;
    Section III-A, Section III-B-2) on the bench mesh for nvec vectors, beside the same call
    on the lumped operator, and one M X.  Any failure is reported in the returned object."""
    import torch

    import workloads
    op2 = None
    try:
        nq = w.p + 2
        op2 = R.rcf_op_create(ctx, prob.mesh)
        R.rcf_op_set_gauss(ctx, op2, nq)
        xq = R.rcf_op_gauss_points(ctx, op2, prob.ncells, nq).reshape(-1, 3)
        prm = prob.params
        V = workloads.gaussian_sum_potential(xq, prm["centres"], prm["depths"], prm["widths"], prm["L"])
        B = workloads.smooth_periodic_field(xq, prm["kvec"], prm["amps"], prm["phases"], prm["L"], prm["bmax"])
        R.rcf_potential_set(ctx, op2, V.reshape(prob.ncells, -1), B.reshape(3, prob.ncells, -1))
        if w.natoms > 0:
            R.rcf_projectors_set(ctx, op2, prm["atoms"], prm["proj_width"], prm["proj_h"])
        N = prob.N
        Zk = torch.randn((nvec, N), dtype=torch.complex64, device=dev, generator=gen)
        Zm = torch.randn((nvec, N), dtype=torch.complex64, device=dev, generator=gen)
        Rr = torch.randn((nvec, N), dtype=torch.complex64, device=dev, generator=gen)
        O = torch.empty_like(Zk)
        g = torch.full((nvec,), 0.25, dtype=torch.float64, device=dev)
        st = lambda o: R.rcf_cheb_step(ctx, o, R.RCF_FORM_H_DINV, R.RCF_FP32, Zk, Zm, Rr, 0.1, -0.5, -1.0, g, O)
        st(op2)
        fm_ms = timed(lambda: st(op2), 5)
        st(prob.op)
        lumped_ms = timed(lambda: st(prob.op), 5)
        R.rcf_mass_apply(ctx, op2, Zk, O, R.RCF_FP32)
        m_ms = timed(lambda: R.rcf_mass_apply(ctx, op2, Zk, O, R.RCF_FP32), 5)
        alg = BYTES_PER_UNIT * N * nvec
        return {"vectors": nvec, "gauss_points_per_direction": nq, "step_ms": fm_ms, "lumped_step_ms": lumped_ms,
                "ratio_to_lumped": fm_ms / lumped_ms, "mass_apply_ms": m_ms,
                "step_algorithmic_gbs": alg / (fm_ms * 1e-3) / 1e9,
                "note": "rcf_cheb_step, FP32, form H D^-1 with the consistent mass (fused x-y pass per plane, "
                        "per-cell Gauss-point potential, z march with the node gather and the combination, "
                        "projectors); algorithmic bytes as the lumped step's (32 B per unit)"}
    except Exception as exc:
        return {"error": repr(exc)[:300]}
    finally:
        if op2 is not None:
            R.rcf_op_destroy(op2)


def run_ours(args):
    import numpy as np
    import torch

    from paper_2605_30128_gb300.build import build as build_library
    from paper_2605_30128_gb300 import rchfsi as R
    from paper_2605_30128_gb300.problem import GPUProblem

    ws, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    if rank == 0:
        build_library()
    barrier(ws)
    w = workload_of(args)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    prob = GPUProblem(w, device=local, stream=stream)
    ctx, op = prob.ctx, prob.op
    N, nvec, q = prob.N, w.nvec, w.degree
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed + 100 + rank)
    X = torch.randn((nvec, N), dtype=torch.complex128, device=dev, generator=gen)
    Y = torch.empty_like(X)
    # filter bounds from a seeded Lanczos run; Ritz values spread below lambda_T
    v0 = torch.randn((N,), dtype=torch.complex128, device=dev, generator=gen)
    lo, hi = R.rcf_lanczos_bounds(ctx, op, w.lanczos, v0)
    lT = lo + 0.05 * (hi - lo)
    ritz = np.linspace(lo, lT, nvec, endpoint=False)
    bounds = (lo - 1e-3 * abs(lo), lT, hi)
    peak = measured_hbm_peak()
    if args.codec_only:
        if rank == 0:
            obj = codec_leg(R, ctx, op, X[:w.block], ritz[:w.block], peak[0], stream)
            print(json.dumps({"bfp_codec": obj, "config": {"workload": describe(w)}}), flush=True)
        prob.close()
        return 0

    def step(prec=R.RCF_FP32):
        R.rcf_filter(ctx, op, X, ritz, q, bounds, R.RCF_RCHFSI, prec, w.block, Y)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        """Average ms of fn over reps calls, CUDA events on the library's stream."""
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    l0 = R.rcf_launch_count(ctx)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(ws)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
    m = {"launches": R.rcf_launch_count(ctx) - l0, "clocks": clk.summary(),
         "ms": max_over_ranks(ws, ev0.elapsed_time(ev1) / args.steps),
         "N": N, "nvec": nvec, "degree": q, "l2_gb": X.numel() * 16 / 1e9, "peak": peak,
         "traffic": traffic_record()}

    # the same filter with the residual in double-float arithmetic, and with the recurrence
    # stored in 16 bits
    def time_variant(prec):
        step(prec)
        barrier(ws)
        return max_over_ranks(ws, timed(lambda: step(prec), max(1, args.steps - 1)))

    m["variants_ms"] = {"df_residual": time_variant(R.RCF_FP32_DF),
                        "fp16_storage": time_variant(R.RCF_FP16),
                        "bf16_storage": time_variant(R.RCF_BF16),
                        "bfp12_residual": time_variant(R.RCF_FP32_BFP12)}

    # ---- dominant kernel: one FP32 recurrence step on a block, timed alone ----
    blk = min(w.block, nvec)
    op1 = R.rcf_op_create(ctx, prob.mesh)       # same mesh and potential, no projectors: one launch
    R.rcf_potential_set(ctx, op1, prob.V, prob.B)
    Zk = torch.randn((blk, N), dtype=torch.complex64, device=dev, generator=gen)
    Zm = torch.randn((blk, N), dtype=torch.complex64, device=dev, generator=gen)
    Rr = torch.randn((blk, N), dtype=torch.complex64, device=dev, generator=gen)
    g = torch.full((blk,), 0.25, dtype=torch.float64, device=dev)
    st = lambda o: R.rcf_cheb_step(ctx, o, R.RCF_FORM_H_DINV, R.RCF_FP32, Zk, Zm, Rr, 0.1, -0.5, -1.0, g, Zm)
    timed(lambda: st(op1), 3)
    kern = {"blk": blk, "k_ms": timed(lambda: st(op1), 10),
            "step_ms": timed(lambda: st(op), 10)}       # with the projectors (four launches)
    # the same step with the vectors stored as binary16 (16 B per unit)
    zk16 = torch.view_as_real(Zk).reshape(blk, -1).to(torch.float16)
    zm16 = torch.view_as_real(Zm).reshape(blk, -1).to(torch.float16)
    rr16 = torch.view_as_real(Rr).reshape(blk, -1).to(torch.float16)
    st16 = lambda: R.rcf_cheb_step(ctx, op1, R.RCF_FORM_H_DINV, R.RCF_FP16, zk16, zm16, rr16,
                                   0.1, -0.5, -1.0, g, zm16)
    timed(st16, 3)
    kern["k16_ms"] = timed(st16, 10)
    del zk16, zm16, rr16
    # the FP32 step reading R from its 12-bit BFP stream (27 B per unit)
    rs = torch.empty((R.rcf_bfp_stream_bytes(4 * (N // 2) * blk, 12),), dtype=torch.uint8, device=dev)
    R.rcf_bfp_encode(ctx, torch.view_as_real(Rr).reshape(-1), 12, rs)
    stb = lambda: R.rcf_cheb_step(ctx, op1, R.RCF_FORM_H_DINV, R.RCF_FP32_BFP12, Zk, Zm, rs,
                                  0.1, -0.5, -1.0, g, Zm)
    timed(stb, 3)
    kern["kbfp_ms"] = timed(stb, 10)
    del rs
    m["kernel"] = kern
    R.rcf_op_destroy(op1)
    del Zk, Zm, Rr
    # the residual of one block: native FP64 (the headline path) and double-float
    R64 = torch.empty((blk, N), dtype=torch.complex128, device=dev)
    R.rcf_residual(ctx, op, X[:blk], ritz[:blk], R64)
    res64 = timed(lambda: R.rcf_residual(ctx, op, X[:blk], ritz[:blk], R64), 1)
    del R64
    Rh = torch.empty((blk, N), dtype=torch.complex64, device=dev)
    R.rcf_residual_df(ctx, op, X[:blk], ritz[:blk], Rh)
    m["residual"] = {"fp64_ms": res64,
                     "df_ms": timed(lambda: R.rcf_residual_df(ctx, op, X[:blk], ritz[:blk], Rh), 1)}
    del Rh

    if not args.no_extras:
        # ---- FP64 ChFSI on one block, same mesh and degree, beside the headline filter ----
        Xb, Yb = X[:blk], Y[:blk]
        f64 = lambda: R.rcf_filter(ctx, op, Xb, ritz[:blk], q, bounds, R.RCF_CHFSI, R.RCF_FP64, blk, Yb)
        mix = lambda: R.rcf_filter(ctx, op, Xb, ritz[:blk], q, bounds, R.RCF_RCHFSI, R.RCF_FP32, blk, Yb)
        f64()
        m["fp64_chfsi"] = {"blk": blk, "f64_ms": timed(f64, 1), "mix_ms": timed(mix, 1)}

        # ---- end to end through the C ABI with host buffers ----
        try:
            Xh = torch.empty((nvec, N), dtype=torch.complex128, pin_memory=True)
            Yh = torch.empty((nvec, N), dtype=torch.complex128, pin_memory=True)
            Xh.copy_(X)
            sample = "full workload"
        except Exception:
            Xh = torch.empty((blk, N), dtype=torch.complex128, pin_memory=True)
            Yh = torch.empty((blk, N), dtype=torch.complex128, pin_memory=True)
            Xh.copy_(X[:blk])
            sample = f"first block of {blk} vectors (pinned host memory for the full block set unavailable)"
        ne = Xh.shape[0]
        # the C ABI's host-buffer filter: band blocks stream through device slots, copies in
        # and out overlapping the filtering of the neighbouring blocks
        host = lambda: R.rcf_filter_host(ctx, op, Xh, ritz[:ne], q, bounds, R.RCF_RCHFSI, R.RCF_FP32, w.block, Yh)
        host()
        torch.cuda.synchronize()
        calls = []
        for _ in range(max(1, args.steps)):
            t0 = time.perf_counter()
            host()
            torch.cuda.synchronize()
            calls.append((time.perf_counter() - t0) * 1e3)
        e_ms = max_over_ranks(ws, sum(calls) / len(calls))
        # the host link of this machine, pinned buffers, one direction at a time (the
        # end-to-end time cannot fall below the larger of the two copy times)
        nl = min(64, ne)
        dbuf = torch.empty((nl, N), dtype=torch.complex128, device=dev)
        link = {}
        for name, dst, src in (("h2d_gbs", dbuf, Xh[:nl]), ("d2h_gbs", Yh[:nl], dbuf)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            link[name] = 3 * dbuf.numel() * 16 / (e0.elapsed_time(e1) * 1e6)
        del dbuf
        m["e2e"] = {"ms": e_ms, "ne": ne, "h2d": Xh.numel() * 16, "d2h": Yh.numel() * 16,
                    "sample": sample, "link": link, "calls_ms": [round(c, 1) for c in calls]}
        del Xh, Yh

        # ---- the adjoint filter on the 8^3-cell p = 4 workload (64 vectors, degree 15,
        #      checkpoints every 5 steps) against its forward filter ----
        wa = workloads_mod().workload("cfg4")
        pa_ = GPUProblem(wa, device=local, stream=stream)
        Xa = torch.randn((wa.nvec, pa_.N), dtype=torch.complex128, device=dev, generator=gen)
        Xa /= torch.linalg.norm(Xa, dim=1, keepdim=True)
        va = torch.randn((pa_.N,), dtype=torch.complex128, device=dev, generator=gen)
        la, ha = R.rcf_lanczos_bounds(pa_.ctx, pa_.op, wa.lanczos, va)
        ra = np.linspace(la, la + 0.05 * (ha - la), wa.nvec, endpoint=False)
        ba = (la - 1e-3 * abs(la), la + 0.05 * (ha - la), ha)
        Ya = torch.empty_like(Xa)
        Ybar = torch.randn_like(Xa)
        dV = torch.zeros((pa_.ncells, pa_.nloc), dtype=torch.float64, device=dev)
        dB = torch.zeros((3, pa_.ncells, pa_.nloc), dtype=torch.float64, device=dev)
        adj = {}
        for pname, prec in (("fp64", R.RCF_FP64), ("fp32", R.RCF_FP32)):
            fwd = lambda: R.rcf_filter(pa_.ctx, pa_.op, Xa, ra, wa.degree, ba, R.RCF_RCHFSI, prec, wa.nvec, Ya)
            bwd = lambda: R.rcf_adjoint_filter(pa_.ctx, pa_.op, Xa, ra, wa.degree, ba, R.RCF_RCHFSI, prec, Ybar,
                                               wa.ckpt, dV, dB, None)
            fwd(); bwd()
            f_ms, b_ms = timed(fwd, 1), timed(bwd, 1)
            adj[pname] = {"forward_ms": f_ms, "adjoint_ms": b_ms, "ratio": b_ms / f_ms}
        m["adjoint"] = dict(adj, workload=describe(wa), note="adjoint w.r.t. V, B at all quadrature "
                            "points, checkpoints every %d steps" % wa.ckpt)
        pa_.close()
        del Xa, Ya, Ybar, dV, dB

        # ---- the periodic Poisson solve on the same mesh (Section III-B-1; Algorithm
        #      pcg_fusion): the matrix-free K x kernel and the fused PCG ----
        m["poisson"] = poisson_leg(R, ctx, prob.mesh, w, dev, gen, timed)

        # ---- the full consistent mass (Section III-A; Section III-B-2): one step ----
        m["fullmass"] = fullmass_leg(R, ctx, prob, w, dev, gen, timed)

        # ---- block floating-point codec (Section III-C-3) on one residual block ----
        m["bfp_codec"] = codec_leg(R, ctx, op, X[:blk], ritz[:blk], peak[0], stream)

        # ---- CPU oracle on a bounded sample (rank 0, one GPU only) ----
        if ws == 1 and rank == 0:
            H = oracle_setup(w)
            v, dt = oracle_sample(H, ORACLE_NV, ORACLE_Q, 700)
            m["cpu_baseline"] = {"value": v, "dt": dt}
    if rank == 0:
        print(json.dumps(assemble_line(w, ws, args.steps, args.warmup, m)), flush=True)
    prob.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
