"""The R-ChFSI property behind the 16-bit storage variants, on the CPU: with Z_k, Z_{k-1} and R
rounded to 16 bits whenever stored (exact FP64 arithmetic otherwise, tests/lowprec_emulation.py),
the filter's error against the oracle's FP64 filter falls in proportion to the residual.  On the
4^3-cell workload near an eigenvector block (perturbations 1e-3 and 1e-6) the errors are about
9.8e-7 / 9.8e-10 (binary16) and 7.0e-6 / 7.0e-9 (bfloat16): the scales the GPU tests of RCF_FP16 /
RCF_BF16 allow with a factor 5.  A 16-bit rounding of the stored vectors alone, without the
residual form (plain ChFSI with 16-bit storage of Y_k), keeps an error near the 16-bit epsilon."""
import numpy as np
import pytest

import workloads
from lowprec_emulation import rchfsi_filter_16, round16
from oracle import chfsi_filter, lanczos_bounds, rayleigh_ritz, rchfsi_eigensolver, rchfsi_filter
from oracle.chebyshev import filter_scalars
from oracle_cases import build_oracle


def test_round16_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.5e-3])
    f16 = round16(x, "fp16").real
    assert f16[1] == 1.0 and f16[2] == 1.0 + 2 ** -9       # ties to even at half a binary16 ulp
    b16 = round16(x, "bf16").real
    assert b16[3] == 1.0 and b16[4] == 1.0 + 2 ** -6       # ties to even at half a bfloat16 ulp
    assert abs(b16[5] + 1.5e-3) <= 2 ** -8 * 1.5e-3         # half an ulp: at most 2^-8 relative
    assert np.all(round16(f16, "fp16").real == f16)         # idempotent


@pytest.fixture(scope="module")
def near_converged():
    w = workloads.workload("cfg1")
    H, *_ = build_oracle(w)
    X, _ = rayleigh_ritz(H, workloads.complex_normal(w.seed + 100, (H.N, w.nvec)))
    v0 = workloads.complex_normal(w.seed + 200, H.N)
    lo, hi, *_ = lanczos_bounds(H, v0, w.lanczos)
    Xc, lam_c, _ = rchfsi_eigensolver(H, X, q=10, lmax=hi, tol=1e-11, max_cycles=80, nwanted=28)
    b = (float(lam_c.min()), float(lam_c.max()), hi)
    return H, Xc, lam_c, b, workloads.complex_normal(77, Xc.shape)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fmt,lo,hi", [("fp16", 4e-7, 2e-6), ("bf16", 3e-6, 1.5e-5)])
def test_16bit_storage_error_is_residual_proportional(near_converged, fmt, lo, hi):
    H, Xc, lam, b, noise = near_converged
    errs = []
    for delta in (1e-3, 1e-6):
        X = Xc + delta * noise / np.linalg.norm(noise) * np.linalg.norm(Xc)
        ref = rchfsi_filter(H, X, lam, *b, 10)
        errs.append(_rel(rchfsi_filter_16(H, X, lam, *b, 10, fmt)[:, :28], ref[:, :28]))
    assert lo < errs[0] < hi
    assert 0.5e-3 < errs[1] / errs[0] < 2e-3                  # scales with the perturbation


def test_16bit_storage_without_residual_form_keeps_its_floor(near_converged):
    """ChFSI with Y_k stored in binary16: the error does not fall with the perturbation."""
    H, Xc, lam, b, noise = near_converged
    c, e, sigma = filter_scalars(*b, 10)
    Minv = 1.0 / H.Mdiag[:, None]
    errs = []
    for delta in (1e-3, 1e-6):
        X = Xc + delta * noise / np.linalg.norm(noise) * np.linalg.norm(Xc)
        ref = chfsi_filter(H, X, *b, 10)
        Yp, Y = round16(X, "fp16"), round16((sigma[1] / e) * (Minv * H.apply(X) - c * X), "fp16")
        for k in range(1, 10):
            a = 2.0 * sigma[k + 1] / e
            Yp, Y = Y, round16(a * (Minv * H.apply(Y) - c * Y) - sigma[k] * sigma[k + 1] * Yp, "fp16")
        errs.append(_rel(Y[:, :28], ref[:, :28]))
    assert errs[1] > 0.3 * errs[0] > 1e-5


# ---- block floating-point storage (Section III-C-3 format, one block per node and vector) ----

def test_bfp_rounding_matches_the_oracle_codec():
    from lowprec_emulation import bfp_round_blocks
    from oracle.bfp import bfp_decode, bfp_encode
    x = workloads.bfp_values(9, 40000)
    for nbits in (16, 12, 10):
        a = bfp_round_blocks(x.reshape(-1, 4), nbits).astype(np.float32).ravel()
        assert np.array_equal(a.view(np.uint32), bfp_decode(bfp_encode(x, nbits), x.size, nbits).view(np.uint32))


@pytest.mark.parametrize("nbits,lo,hi", [(16, 1.5e-7, 7e-7), (12, 2.5e-6, 1.1e-5), (10, 1e-5, 4.5e-5)])
def test_bfp_storage_error_is_residual_proportional(near_converged, nbits, lo, hi):
    """Z_k, Z_{k-1} and R stored in BFP: measured 3.5e-7 / 5.5e-6 / 2.2e-5 at a 1e-3 perturbation
    (16 / 12 / 10 bits; binary16 gives 9.8e-7, bfloat16 7.0e-6), falling 1000x with it."""
    from lowprec_emulation import rchfsi_filter_bfp
    H, Xc, lam, b, noise = near_converged
    errs = []
    for delta in (1e-3, 1e-6):
        X = Xc + delta * noise / np.linalg.norm(noise) * np.linalg.norm(Xc)
        ref = rchfsi_filter(H, X, lam, *b, 10)
        errs.append(_rel(rchfsi_filter_bfp(H, X, lam, *b, 10, nbits)[:, :28], ref[:, :28]))
    assert lo < errs[0] < hi
    assert 0.5e-3 < errs[1] / errs[0] < 2e-3


@pytest.mark.parametrize("nbits,lo,hi", [(16, 1.2e-7, 6e-7), (12, 2e-6, 9e-6)])
def test_bfp_residual_storage_error_is_residual_proportional(near_converged, nbits, lo, hi):
    """R alone stored in BFP (the library's RCF_FP32_BFP12 at 12 bits): measured 2.7e-7 / 4.4e-6
    at a 1e-3 perturbation (16 / 12 bits), falling 1000x with it; most of the error of storing
    Z_k, Z_{k-1} and R comes from R, the term every step adds."""
    from lowprec_emulation import rchfsi_filter_bfp, rchfsi_filter_bfp_residual
    H, Xc, lam, b, noise = near_converged
    errs, full = [], []
    for delta in (1e-3, 1e-6):
        X = Xc + delta * noise / np.linalg.norm(noise) * np.linalg.norm(Xc)
        ref = rchfsi_filter(H, X, lam, *b, 10)
        errs.append(_rel(rchfsi_filter_bfp_residual(H, X, lam, *b, 10, nbits)[:, :28], ref[:, :28]))
        full.append(_rel(rchfsi_filter_bfp(H, X, lam, *b, 10, nbits)[:, :28], ref[:, :28]))
    assert lo < errs[0] < hi
    assert 0.5e-3 < errs[1] / errs[0] < 2e-3
    assert 0.5 * full[0] < errs[0] < full[0]


def test_bfp_storage_eigensolver_follows_the_fp64_loop(near_converged):
    """Algorithm 1 from a perturbed block: with 12-bit BFP storage the residual history and the
    Ritz values follow the FP64 filter's, cycle by cycle."""
    from lowprec_emulation import rchfsi_filter_bfp
    from oracle import residual
    H, Xc, lam_c, b, noise = near_converged
    X0 = Xc + 1e-3 * noise / np.linalg.norm(noise) * np.linalg.norm(Xc)
    runs = {}
    for name in ("fp64", "bfp12"):
        X, lam = rayleigh_ritz(H, X0)
        hist = []
        for _ in range(8):
            hist.append(np.linalg.norm(residual(H, X, lam), axis=0)[:28].max())
            if name == "fp64":
                Y = rchfsi_filter(H, X, lam, float(lam.min()), float(lam.max()), b[2], 10)
            else:
                Y = rchfsi_filter_bfp(H, X, lam, float(lam.min()), float(lam.max()), b[2], 10, 12)
            X, lam = rayleigh_ritz(H, Y)
        runs[name] = (np.array(hist), lam)
    h64, hb = runs["fp64"][0], runs["bfp12"][0]
    assert h64[-1] < 0.2 * h64[0]
    np.testing.assert_allclose(hb, h64, rtol=1e-3)
    np.testing.assert_allclose(runs["bfp12"][1][:28], runs["fp64"][1][:28], atol=1e-9)


# ---- mixed-precision subspace rotation (Section III-C-4) ----

def _loop(H, X0, rr, cycles, hi):
    from oracle import residual
    X, lam = rayleigh_ritz(H, X0)
    hist = []
    for _ in range(cycles):
        hist.append(np.linalg.norm(residual(H, X, lam), axis=0)[:28].max())
        Y = rchfsi_filter(H, X, lam, float(lam.min()), float(lam.max()), hi, 10)
        X, lam = rr(H, Y)
    return np.array(hist), lam


def test_mixed_precision_rotation_follows_the_fp64_loop(near_converged):
    """X = Y Q_diag (FP64) + Y Q_offdiag (FP32): from the start block and from a converged block,
    Algorithm 1's residual history and Ritz values match the all-FP64 rotation."""
    from lowprec_emulation import rayleigh_ritz_mixed_rotation
    H, Xc, lam_c, b, _ = near_converged
    w = workloads.workload("cfg1")
    X0 = workloads.complex_normal(w.seed + 100, (H.N, w.nvec))
    for start, cycles, rtol in ((X0, 16, 1e-6), (Xc, 6, 1e-3)):
        h64, l64 = _loop(H, start, rayleigh_ritz, cycles, b[2])
        hmx, lmx = _loop(H, start, rayleigh_ritz_mixed_rotation, cycles, b[2])
        assert h64[-1] < h64[0]
        np.testing.assert_allclose(hmx, h64, rtol=rtol)
        np.testing.assert_allclose(lmx[:28], l64[:28], atol=1e-12)
