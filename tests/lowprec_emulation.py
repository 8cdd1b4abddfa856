"""CPU emulation of the R-ChFSI filter with its recurrence vectors stored in 16 bits or in the
block floating-point format of Section III-C-3 (test helper).

Z_k, Z_{k-1} and R are rounded to binary16 / bfloat16 (round to nearest even) each time they are
stored, R scaled per column by the power of two that puts its largest entry in [1/2, 1); the
arithmetic is FP64, so the difference from the oracle's filter is the storage rounding alone.
It mirrors the recurrence of the library's RCF_FP16 / RCF_BF16 filters and is the source of the
error scales their GPU tests allow (it uses the oracle's building blocks, not the GPU code).
"""
import numpy as np

from oracle.chebyshev import filter_scalars, ritz_filter_values


def round16(x: np.ndarray, fmt: str) -> np.ndarray:
    """Real and imaginary parts rounded to binary16 ('fp16') or bfloat16 ('bf16')."""
    def one(a):
        if fmt == "fp16":
            return a.astype(np.float16).astype(np.float64)
        f = a.astype(np.float32)
        b = f.view(np.uint32).astype(np.uint64)
        b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)   # RNE to the top 16 bits
        return b.view(np.float32).astype(np.float64)
    return one(np.real(x)) + 1j * one(np.imag(x))


def rchfsi_filter_16(Hop, X, lam, lmin, lT, lmax, q, fmt):
    c, e, sigma = filter_scalars(lmin, lT, lmax, q)
    lam = np.asarray(lam, dtype=np.float64)
    Dinv = 1.0 / Hop.Mdiag[:, None]
    R = Hop.apply(X) - Hop.Mdiag[:, None] * X * lam[None, :]
    m = np.max(np.maximum(np.abs(R.real), np.abs(R.imag)), axis=0)
    s = np.where(m > 0, 2.0 ** (np.floor(np.log2(np.where(m > 0, m, 1.0))) + 1), 1.0)
    Rs = round16(R / s[None, :], fmt)
    Lk = ritz_filter_values(lam, lmin, lT, lmax, q)
    Zprev, Z = np.zeros_like(X), round16((sigma[1] / e) * Rs, fmt)
    for k in range(1, q):
        a = 2.0 * sigma[k + 1] / e
        Zn = a * Hop.apply(Dinv * Z) - a * c * Z - sigma[k] * sigma[k + 1] * Zprev + a * Rs * Lk[k][None, :]
        Zprev, Z = Z, round16(Zn, fmt)
    return Dinv * Z * s[None, :] + X * Lk[q][None, :]


def bfp_round(x: np.ndarray, nbits: int) -> np.ndarray:
    """Complex (2M, nvec) multivector rounded to FP32 and then through the block floating-point
    format of Section III-C-3, one block per node and vector: the node's (re_up, im_up, re_dn,
    im_dn).  Vectorised restatement of oracle.bfp (checked against it bit for bit)."""
    v = nbits - 2
    x = np.asarray(x)
    n2, nv = x.shape
    r = np.empty((n2 // 2, 4, nv), dtype=np.float32)
    r[:, 0], r[:, 1] = x[0::2].real, x[0::2].imag
    r[:, 2], r[:, 3] = x[1::2].real, x[1::2].imag
    y = bfp_round_blocks(r.transpose(0, 2, 1).reshape(-1, 4), nbits).reshape(n2 // 2, nv, 4)
    out = np.empty_like(x, dtype=np.complex128)
    out[0::2] = y[:, :, 0] + 1j * y[:, :, 1]
    out[1::2] = y[:, :, 2] + 1j * y[:, :, 3]
    return out


def bfp_round_blocks(b: np.ndarray, nbits: int) -> np.ndarray:
    """(nblocks, 4) float32 -> the decoded values of their BFP encoding (float64)."""
    v = nbits - 2
    b = np.asarray(b, dtype=np.float32).astype(np.float64)
    m = np.abs(b).max(axis=1)
    _, ex = np.frexp(np.where(m > 0, m, 1.0))
    emax = np.maximum(ex, -126)
    qmax = 2.0 ** (v - 1) - 1
    q = np.rint(np.ldexp(b, (v - 1 - emax)[:, None])) + 0.0     # integer coefficients: no -0
    q = np.minimum(q, qmax)
    q = np.where((emax == 128)[:, None], np.maximum(q, -qmax), q)
    y = np.ldexp(q, (emax - v + 1)[:, None])
    return np.where((m > 0)[:, None], y, 0.0)


def rchfsi_filter_bfp(Hop, X, lam, lmin, lT, lmax, q, nbits):
    """R-ChFSI with Z_k, Z_{k-1} and R stored in BFP at nbits per value (FP64 arithmetic)."""
    c, e, sigma = filter_scalars(lmin, lT, lmax, q)
    lam = np.asarray(lam, dtype=np.float64)
    Dinv = 1.0 / Hop.Mdiag[:, None]
    R = Hop.apply(X) - Hop.Mdiag[:, None] * X * lam[None, :]
    Rs = bfp_round(R, nbits)
    Lk = ritz_filter_values(lam, lmin, lT, lmax, q)
    Zprev, Z = np.zeros_like(X), bfp_round((sigma[1] / e) * Rs, nbits)
    for k in range(1, q):
        a = 2.0 * sigma[k + 1] / e
        Zn = a * Hop.apply(Dinv * Z) - a * c * Z - sigma[k] * sigma[k + 1] * Zprev + a * Rs * Lk[k][None, :]
        Zprev, Z = Z, bfp_round(Zn, nbits)
    return Dinv * Z + X * Lk[q][None, :]


def rchfsi_filter_bfp_residual(Hop, X, lam, lmin, lT, lmax, q, nbits=12):
    """R-ChFSI with R alone stored in BFP (its FP32 rounding through the format; every use of R
    sees the decoded values) and Z_k exact (FP64 arithmetic): the reference of the library's
    RCF_FP32_BFP12, whose remaining difference from it is the FP32 recurrence."""
    from oracle.filters import residual
    c, e, sigma = filter_scalars(lmin, lT, lmax, q)
    Dinv = 1.0 / Hop.Mdiag[:, None]
    Rt = bfp_round(residual(Hop, X, lam), nbits)
    Lk = ritz_filter_values(np.asarray(lam, dtype=np.float64), lmin, lT, lmax, q)
    Zp, Z = np.zeros_like(Rt), (sigma[1] / e) * Rt
    for k in range(1, q):
        a = 2.0 * sigma[k + 1] / e
        Zp, Z = Z, a * Hop.apply(Dinv * Z) - a * c * Z - sigma[k] * sigma[k + 1] * Zp + a * Rt * Lk[k][None, :]
    return Dinv * Z + X * Lk[q][None, :]


def rayleigh_ritz_mixed_rotation(Hop, Y):
    """Rayleigh-Ritz whose subspace rotation X = Y Q is split as in Section III-C-4:
    Y Q_diag in FP64 plus Y Q_offdiag in FP32 (complex64 operands and products, rounded
    back), Q_diag the diagonal of Q."""
    from oracle.rr import cholqr2
    Yo = cholqr2(Y, Hop.Mdiag)
    A = Yo.conj().T @ Hop.apply(Yo)
    A = 0.5 * (A + A.conj().T)
    theta, Q = np.linalg.eigh(A)
    Qd = np.diag(np.diag(Q))
    Xo = (Yo.astype(np.complex64) @ (Q - Qd).astype(np.complex64)).astype(np.complex128)
    return Yo @ Qd + Xo, theta


def rchfsi_filter_fp32(Hop, X, lam, lmin, lT, lmax, q):
    """R-ChFSI with the recurrence in FP32 (complex64 Z_k, Z_{k-1}, R; each product H D^-1 Z_k
    rounded to FP32), the residual R = H X - M X Lambda in FP64 with the operator's own M
    (the full mass where it has one) and D^-1 = 1 / Mdiag: Section III-C's split, on any
    operator of the oracle."""
    from oracle.filters import residual
    c, e, sigma = filter_scalars(lmin, lT, lmax, q)
    Dinv = 1.0 / Hop.Mdiag[:, None]
    R32 = residual(Hop, X, lam).astype(np.complex64)
    Lk = ritz_filter_values(np.asarray(lam, dtype=np.float64), lmin, lT, lmax, q)
    Zp, Z = np.zeros_like(R32), ((sigma[1] / e) * R32).astype(np.complex64)
    for k in range(1, q):
        a = 2.0 * sigma[k + 1] / e
        HZ = Hop.apply(Dinv * Z.astype(np.complex128)).astype(np.complex64)
        Zn = (np.float32(a) * HZ - np.float32(a * c) * Z - np.float32(sigma[k] * sigma[k + 1]) * Zp
              + np.float32(a) * R32 * Lk[k][None, :].astype(np.float32))
        Zp, Z = Z, Zn.astype(np.complex64)
    return Dinv * Z.astype(np.complex128) + X * Lk[q][None, :]
