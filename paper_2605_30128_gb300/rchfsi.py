"""Thin ctypes binding of librchfsi (include/rchfsi.h), same names as the C ABI.

Only argument marshalling happens here: every step of the computation runs in
the library's CUDA kernels.  Device multivectors are torch tensors of shape
(nvec, 2M) (row j = vector j, so the memory is the column-major layout of
the C ABI), dtype complex128 (or complex64 where the C call accepts FP32).
If the library is missing, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librchfsi.so")

RCF_OK, RCF_EINVAL, RCF_ENOMEM, RCF_ECUDA, RCF_ENOTSPD, RCF_ETIMEOUT, RCF_ENOTSUP = range(7)
RCF_FP64, RCF_FP32, RCF_FP32_DF, RCF_FP16, RCF_BF16, RCF_FP32_BFP12 = 0, 1, 2, 3, 4, 5
RCF_CHFSI, RCF_RCHFSI = 0, 1
RCF_FORM_H, RCF_FORM_DINV_H, RCF_FORM_H_DINV = 0, 1, 2
RCF_STEP_CPASYNC, RCF_STEP_TMA = 0, 1
RCF_RR_FP64, RCF_RR_DF, RCF_RR_TC, RCF_RR_MIXED = 0, 1, 2, 3

EXPORTS = [
    "rcf_create", "rcf_destroy", "rcf_status_string", "rcf_last_error", "rcf_sync",
    "rcf_mesh_create", "rcf_mesh_destroy", "rcf_mesh_info", "rcf_mesh_connectivity",
    "rcf_mesh_quadrature_points", "rcf_mesh_mass", "rcf_op_create", "rcf_op_destroy",
    "rcf_potential_set", "rcf_projectors_set", "rcf_projectors_couplings", "rcf_projector_support",
    "rcf_apply", "rcf_lanczos_bounds", "rcf_residual", "rcf_filter", "rcf_rayleigh_ritz",
    "rcf_grad_bilinear", "rcf_adjoint_filter", "rcf_cheb_step", "rcf_launch_count",
    "rcf_apply_noalloc", "rcf_set_step_kernel", "rcf_residual_df", "rcf_cholqr2",
    "rcf_rayleigh_ritz_orth", "rcf_filter_host", "rcf_set_rr_arith",
    "rcf_bfp_stream_bytes", "rcf_bfp_encode", "rcf_bfp_decode", "rcf_ritz_cotangent",
    "rcf_set_wait_limit", "rcf_inner", "rcf_rotate", "rcf_laplacian", "rcf_poisson_pcg", "rcf_workspace_bytes",
    "rcf_op_set_gauss", "rcf_op_gauss_points", "rcf_mass_apply",
]

_lib = None


class RcfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rcf status {status}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load librchfsi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2605_30128_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    pvp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "rcf_create": (i32, [pvp, i32, vp]),
        "rcf_destroy": (i32, [vp]),
        "rcf_status_string": (ctypes.c_char_p, [i32]),
        "rcf_last_error": (ctypes.c_char_p, [vp]),
        "rcf_sync": (i32, [vp]),
        "rcf_mesh_create": (i32, [vp, vp, vp, i32, pvp]),
        "rcf_mesh_destroy": (i32, [vp]),
        "rcf_mesh_info": (i32, [vp, vp, vp, vp]),
        "rcf_mesh_connectivity": (i32, [vp, vp]),
        "rcf_mesh_quadrature_points": (i32, [vp, vp]),
        "rcf_mesh_mass": (i32, [vp, vp]),
        "rcf_op_create": (i32, [vp, vp, pvp]),
        "rcf_op_destroy": (i32, [vp]),
        "rcf_potential_set": (i32, [vp, vp, vp, i32]),
        "rcf_projectors_set": (i32, [vp, i32, vp, vp, vp, dbl]),
        "rcf_projectors_couplings": (i32, [vp, vp]),
        "rcf_projector_support": (i32, [vp, i32, vp, vp]),
        "rcf_apply": (i32, [vp, vp, i32, vp, i64, i32, vp, i64, i32]),
        "rcf_lanczos_bounds": (i32, [vp, vp, i32, vp, vp, vp]),
        "rcf_residual": (i32, [vp, vp, vp, i64, i32, vp, vp, i64, vp]),
        "rcf_filter": (i32, [vp, vp, vp, i64, i32, vp, i32, vp, i32, i32, i32, vp, i64]),
        "rcf_rayleigh_ritz": (i32, [vp, vp, vp, i64, i32, vp, i64, vp]),
        "rcf_grad_bilinear": (i32, [vp, vp, vp, i64, vp, i64, i32, dbl, vp, vp, vp]),
        "rcf_adjoint_filter": (i32, [vp, vp, vp, i64, i32, vp, i32, vp, i32, i32, vp, i64, i32, vp, vp, vp]),
        "rcf_cheb_step": (i32, [vp, vp, i32, i32, vp, vp, vp, i64, i32, dbl, dbl, dbl, vp, vp]),
        "rcf_launch_count": (i64, [vp]),
        "rcf_apply_noalloc": (i32, [vp, vp, i32, vp, i64, i32, vp, i64, i32]),
        "rcf_set_step_kernel": (i32, [vp, i32]),
        "rcf_set_rr_arith": (i32, [vp, i32]),
        "rcf_residual_df": (i32, [vp, vp, vp, i64, i32, vp, vp, vp, i64]),
        "rcf_cholqr2": (i32, [vp, vp, vp, i64, i32]),
        "rcf_filter_host": (i32, [vp, vp, vp, i64, i32, vp, i32, vp, i32, i32, i32, vp, i64]),
        "rcf_rayleigh_ritz_orth": (i32, [vp, vp, vp, i64, i32, vp, i64, vp]),
        "rcf_bfp_stream_bytes": (i64, [i64, i32]),
        "rcf_bfp_encode": (i32, [vp, vp, i64, i32, vp]),
        "rcf_bfp_decode": (i32, [vp, vp, i64, i32, vp]),
        "rcf_set_wait_limit": (i32, [vp, i64]),
        "rcf_laplacian": (i32, [vp, vp, vp, vp]),
        "rcf_workspace_bytes": (i64, [vp]),
        "rcf_op_set_gauss": (i32, [vp, i32]),
        "rcf_op_gauss_points": (i32, [vp, vp]),
        "rcf_mass_apply": (i32, [vp, vp, vp, i64, i32, vp, i64, i32]),
        "rcf_poisson_pcg": (i32, [vp, vp, vp, vp, i32, dbl, dbl, dbl, i32, vp, vp]),
        "rcf_inner": (i32, [vp, vp, i64, i32, vp, i64, i32, i64, vp, vp, i64, i32]),
        "rcf_rotate": (i32, [vp, vp, i64, i32, vp, i64, i64, vp, i64, i32]),
        "rcf_ritz_cotangent": (i32, [vp, vp, vp, i64, vp, i64, i32, vp, vp, vp, i64, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(ctx, status: int):
    if status != RCF_OK:
        L = lib()
        msg = L.rcf_last_error(ctx).decode() if ctx else L.rcf_status_string(status).decode()
        raise RcfError(status, msg or L.rcf_status_string(status).decode())


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev(t, dtype=None, name="tensor"):
    """(pointer, ld) of a device multivector tensor of shape (nvec, rows)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() == 1:
        return ctypes.c_void_p(t.data_ptr()), t.shape[0]
    if t.stride(-1) != 1:
        raise ValueError(f"{name} rows must be contiguous")
    return ctypes.c_void_p(t.data_ptr()), t.stride(0)


# ---- context / mesh / operator ---------------------------------------------------

def rcf_create(device: int = 0, stream=None):
    """Context on `device`, enqueueing on `stream` (a torch.cuda.Stream, an int handle or None
    for torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = ctypes.c_void_p()
    _check(None, lib().rcf_create(ctypes.byref(h), device, ctypes.c_void_p(stream)))
    return h


def rcf_destroy(ctx):
    lib().rcf_destroy(ctx)


def rcf_sync(ctx):
    _check(ctx, lib().rcf_sync(ctx))


def rcf_status_string(status: int) -> str:
    return lib().rcf_status_string(status).decode()


def rcf_last_error(ctx) -> str:
    return lib().rcf_last_error(ctx).decode()


def rcf_mesh_create(ctx, ncell, side, p: int):
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(ncell, dtype=np.int32), (3,)))
    s = np.ascontiguousarray(np.broadcast_to(np.asarray(side, dtype=np.float64), (3,)))
    h = ctypes.c_void_p()
    _check(ctx, lib().rcf_mesh_create(ctx, _np_ptr(n), _np_ptr(s), int(p), ctypes.byref(h)))
    return h


def rcf_mesh_destroy(mesh):
    lib().rcf_mesh_destroy(mesh)


def rcf_mesh_info(mesh):
    nn, nc, nl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(None, lib().rcf_mesh_info(mesh, ctypes.byref(nn), ctypes.byref(nc), ctypes.byref(nl)))
    return nn.value, nc.value, nl.value


def rcf_mesh_connectivity(mesh) -> np.ndarray:
    nn, nc, nl = rcf_mesh_info(mesh)
    out = np.empty((nc, nl), dtype=np.int32)
    _check(None, lib().rcf_mesh_connectivity(mesh, _np_ptr(out)))
    return out


def rcf_mesh_quadrature_points(mesh) -> np.ndarray:
    nn, nc, nl = rcf_mesh_info(mesh)
    out = np.empty((nc, nl, 3), dtype=np.float64)
    _check(None, lib().rcf_mesh_quadrature_points(mesh, _np_ptr(out)))
    return out


def rcf_mesh_mass(mesh) -> np.ndarray:
    nn, nc, nl = rcf_mesh_info(mesh)
    out = np.empty(nn, dtype=np.float64)
    _check(None, lib().rcf_mesh_mass(mesh, _np_ptr(out)))
    return out


def rcf_op_create(ctx, mesh):
    h = ctypes.c_void_p()
    _check(ctx, lib().rcf_op_create(ctx, mesh, ctypes.byref(h)))
    return h


def rcf_op_destroy(op):
    lib().rcf_op_destroy(op)


def rcf_potential_set(ctx, op, V, B=None):
    """V: [ncells][nloc], B: [3][ncells][nloc] FP64, numpy (host) or CUDA tensors (device)."""
    import torch
    if isinstance(V, torch.Tensor):
        if V.dtype != torch.float64 or not V.is_cuda or not V.is_contiguous():
            raise TypeError("V must be a contiguous float64 CUDA tensor")
        if B is not None and (B.dtype != torch.float64 or not B.is_cuda or not B.is_contiguous()):
            raise TypeError("B must be a contiguous float64 CUDA tensor")
        _check(ctx, lib().rcf_potential_set(op, ctypes.c_void_p(V.data_ptr()),
                                            ctypes.c_void_p(B.data_ptr()) if B is not None else None, 1))
        return
    Vh = np.ascontiguousarray(V, dtype=np.float64)
    Bh = None if B is None else np.ascontiguousarray(B, dtype=np.float64)
    _check(ctx, lib().rcf_potential_set(op, _np_ptr(Vh), _np_ptr(Bh) if Bh is not None else None, 0))


def rcf_projectors_set(ctx, op, pos, width, h, rcut_factor: float = 5.0):
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    width = np.ascontiguousarray(width, dtype=np.float64).reshape(-1, 2)
    h = np.ascontiguousarray(h, dtype=np.float64).reshape(-1, 2)
    _check(ctx, lib().rcf_projectors_set(op, pos.shape[0], _np_ptr(pos), _np_ptr(width), _np_ptr(h),
                                         float(rcut_factor)))


def rcf_projectors_couplings(ctx, op, h):
    h = np.ascontiguousarray(h, dtype=np.float64).reshape(-1, 2)
    _check(ctx, lib().rcf_projectors_couplings(op, _np_ptr(h)))


def rcf_projector_support(op, atom: int) -> np.ndarray:
    n = ctypes.c_int64()
    _check(None, lib().rcf_projector_support(op, atom, ctypes.byref(n), None))
    out = np.empty(n.value, dtype=np.int32)
    _check(None, lib().rcf_projector_support(op, atom, ctypes.byref(n), _np_ptr(out)))
    return out


# ---- compute -----------------------------------------------------------------------

def _dev_mv(t, prec: int, name: str):
    """(pointer, ld in complex elements) of a device multivector of precision prec: complex128
    (FP64), complex64 (FP32), complex32 or float16 with interleaved (re, im) (FP16), bfloat16
    with interleaved (re, im) (BF16); shape (nvec, rows) for complex, (nvec, 2 rows) for real."""
    import torch
    if prec == RCF_FP64:
        return _dev(t, torch.complex128, name)
    if prec in (RCF_FP32, RCF_FP32_BFP12):
        return _dev(t, torch.complex64, name)
    if prec == RCF_FP16 and t.dtype == torch.complex32:
        return _dev(t, torch.complex32, name)
    dt = torch.float16 if prec == RCF_FP16 else torch.bfloat16
    p, ld = _dev(t, dt, name)
    if t.dim() == 2 and ld % 2:
        raise ValueError(f"{name}: interleaved (re, im) rows need an even row stride")
    return p, ld // 2 if t.dim() == 2 else ld // 2


def rcf_apply(ctx, op, form: int, X, Y, prec: int = RCF_FP64):
    px, ldx = _dev_mv(X, prec, "X")
    py, ldy = _dev_mv(Y, prec, "Y")
    nvec = X.shape[0] if X.dim() == 2 else 1
    _check(ctx, lib().rcf_apply(ctx, op, form, px, ldx, nvec, py, ldy, prec))


def rcf_lanczos_bounds(ctx, op, nsteps: int, v0):
    import torch
    pv, _ = _dev(v0, torch.complex128, "v0")
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().rcf_lanczos_bounds(ctx, op, int(nsteps), pv, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def rcf_residual(ctx, op, X, ritz, R=None, colnorm=None):
    import torch
    px, ldx = _dev(X, torch.complex128, "X")
    rz = np.ascontiguousarray(ritz, dtype=np.float64)
    pr, ldr = (None, 0) if R is None else _dev(R, torch.complex128, "R")
    pc = None if colnorm is None else ctypes.c_void_p(colnorm.data_ptr())
    _check(ctx, lib().rcf_residual(ctx, op, px, ldx, X.shape[0], _np_ptr(rz), pr, ldr, pc))


def rcf_residual_df(ctx, op, X, ritz, Rh, Rl=None):
    """Double-float residual: Rh (complex64) = FP32 rounding of H X - M X diag(ritz), Rl the
    remainder (complex64, optional; same leading dimension as Rh)."""
    import torch
    px, ldx = _dev(X, torch.complex128, "X")
    rz = np.ascontiguousarray(ritz, dtype=np.float64)
    ph, ldr = _dev(Rh, torch.complex64, "Rh")
    pl = None
    if Rl is not None:
        pl, ldl = _dev(Rl, torch.complex64, "Rl")
        if ldl != ldr:
            raise ValueError("Rh and Rl must share the leading dimension")
    _check(ctx, lib().rcf_residual_df(ctx, op, px, ldx, X.shape[0], _np_ptr(rz), ph, pl, ldr))


def rcf_filter(ctx, op, X, ritz, degree: int, bounds, mode: int, prec: int, block: int, Y):
    import torch
    px, ldx = _dev(X, torch.complex128, "X")
    py, ldy = _dev(Y, torch.complex128, "Y")
    rz = None if ritz is None else np.ascontiguousarray(ritz, dtype=np.float64)
    b = np.ascontiguousarray(bounds, dtype=np.float64)
    _check(ctx, lib().rcf_filter(ctx, op, px, ldx, X.shape[0], _np_ptr(rz) if rz is not None else None,
                                 int(degree), _np_ptr(b), int(mode), int(prec), int(block), py, ldy))


def _host(t, name):
    """(pointer, ld) of a host multivector tensor of shape (nvec, rows), complex128."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host tensor")
    if t.dtype != torch.complex128:
        raise TypeError(f"{name} must be complex128, got {t.dtype}")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be (nvec, rows) with unit row stride")
    return ctypes.c_void_p(t.data_ptr()), int(t.stride(0))


def rcf_filter_host(ctx, op, X, ritz, degree: int, bounds, mode: int, prec: int, block: int, Y):
    """rcf_filter with X and Y in host memory (pin them for copy/compute overlap)."""
    px, ldx = _host(X, "X")
    py, ldy = _host(Y, "Y")
    rz = None if ritz is None else np.ascontiguousarray(ritz, dtype=np.float64)
    b = np.ascontiguousarray(bounds, dtype=np.float64)
    _check(ctx, lib().rcf_filter_host(ctx, op, px, ldx, X.shape[0], _np_ptr(rz) if rz is not None else None,
                                      int(degree), _np_ptr(b), int(mode), int(prec), int(block), py, ldy))


def rcf_rayleigh_ritz(ctx, op, Y, X_out):
    import torch
    py, ldy = _dev(Y, torch.complex128, "Y")
    px, ldx = _dev(X_out, torch.complex128, "X_out")
    ritz = np.empty(Y.shape[0], dtype=np.float64)
    _check(ctx, lib().rcf_rayleigh_ritz(ctx, op, py, ldy, Y.shape[0], px, ldx, _np_ptr(ritz)))
    return ritz


def rcf_cholqr2(ctx, op, Y):
    """Y (complex128, in/out) made M-orthonormal (Cholesky-QR2)."""
    import torch
    py, ldy = _dev(Y, torch.complex128, "Y")
    _check(ctx, lib().rcf_cholqr2(ctx, op, py, ldy, Y.shape[0]))


def rcf_rayleigh_ritz_orth(ctx, op, Y, X_out):
    """Rayleigh-Ritz on an M-orthonormal Y: Ritz vectors into X_out, Ritz values returned."""
    import torch
    py, ldy = _dev(Y, torch.complex128, "Y")
    px, ldx = _dev(X_out, torch.complex128, "X_out")
    ritz = np.empty(Y.shape[0], dtype=np.float64)
    _check(ctx, lib().rcf_rayleigh_ritz_orth(ctx, op, py, ldy, Y.shape[0], px, ldx, _np_ptr(ritz)))
    return ritz


def rcf_grad_bilinear(ctx, op, W, U, weight: float, dV, dB, dh=None):
    import torch
    pw, ldw = _dev(W, torch.complex128, "W")
    pu, ldu = _dev(U, torch.complex128, "U")
    _check(ctx, lib().rcf_grad_bilinear(ctx, op, pw, ldw, pu, ldu, W.shape[0], float(weight),
                                        ctypes.c_void_p(dV.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
                                        _np_ptr(dh) if dh is not None else None))


def rcf_ritz_cotangent(ctx, op, Y, X, theta, thetabar, Ybar, dV=None, dB=None, dh=None):
    """Ybar <- dL/dY of L = sum_j thetabar_j theta_j(Y) for the Rayleigh-Ritz pairs (theta, X = Y Q)
    of Y; dV, dB (device) and dh (host) += the direct derivative sum_j thetabar_j x_j^H dH x_j."""
    import torch
    py, ldy = _dev(Y, torch.complex128, "Y")
    px, ldx = _dev(X, torch.complex128, "X")
    pb, ldb = _dev(Ybar, torch.complex128, "Ybar")
    th = np.ascontiguousarray(theta, dtype=np.float64)
    tb = np.ascontiguousarray(thetabar, dtype=np.float64)
    n = Y.shape[0]
    if X.shape[0] != n or Ybar.shape[0] != n or th.size != n or tb.size != n:
        raise ValueError("Y, X, Ybar, theta and thetabar must have the same number of vectors")
    _check(ctx, lib().rcf_ritz_cotangent(ctx, op, py, ldy, px, ldx, n, _np_ptr(th), _np_ptr(tb), pb, ldb,
                                         ctypes.c_void_p(dV.data_ptr()) if dV is not None else None,
                                         ctypes.c_void_p(dB.data_ptr()) if dB is not None else None,
                                         _np_ptr(dh) if dh is not None else None))


def rcf_adjoint_filter(ctx, op, X, ritz, degree: int, bounds, mode: int, prec: int, Ybar,
                       ckpt_every: int, dV, dB, dh=None):
    import torch
    px, ldx = _dev(X, torch.complex128, "X")
    pyb, ldyb = _dev(Ybar, torch.complex128, "Ybar")
    rz = np.ascontiguousarray(ritz, dtype=np.float64)
    b = np.ascontiguousarray(bounds, dtype=np.float64)
    _check(ctx, lib().rcf_adjoint_filter(ctx, op, px, ldx, X.shape[0], _np_ptr(rz), int(degree), _np_ptr(b),
                                         int(mode), int(prec), pyb, ldyb, int(ckpt_every),
                                         ctypes.c_void_p(dV.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
                                         _np_ptr(dh) if dh is not None else None))


def rcf_cheb_step(ctx, op, form: int, prec: int, Zk, Zkm1, R, alpha: float, beta: float, gamma: float,
                  g, out):
    """out = alpha op(Zk) + beta Zk + gamma Zkm1 + g[v] R (tensors of shape (nvec, rows)).
    prec RCF_FP32_BFP12: Zk, Zkm1, out complex64 and R a uint8 CUDA tensor holding the 12-bit
    BFP stream of the nvec columns (6 bytes per node and column, column after column)."""
    import torch
    pz, ld = _dev_mv(Zk, prec, "Zk")
    po, ldo = _dev_mv(out, prec, "out")
    if ldo != ld:
        raise ValueError("Zk and out must share the leading dimension")
    pm = None if Zkm1 is None else _dev_mv(Zkm1, prec, "Zkm1")[0]
    if R is not None and prec == RCF_FP32_BFP12:
        need = 6 * (Zk.shape[-1] // 2) * Zk.shape[0]
        if not (R.is_cuda and R.dtype == torch.uint8 and R.is_contiguous() and R.numel() >= need):
            raise ValueError(f"R: a contiguous uint8 CUDA stream of at least {need} bytes is required")
        pr = ctypes.c_void_p(R.data_ptr())
    else:
        pr = None if R is None else _dev_mv(R, prec, "R")[0]
    pg = None if g is None else ctypes.c_void_p(g.data_ptr())
    _check(ctx, lib().rcf_cheb_step(ctx, op, int(form), int(prec), pz, pm, pr, ld, Zk.shape[0],
                                    float(alpha), float(beta), float(gamma), pg, po))


def rcf_launch_count(ctx) -> int:
    return int(lib().rcf_launch_count(ctx))


def rcf_set_rr_arith(ctx, kind: int) -> None:
    """Tall products of Cholesky-QR and Rayleigh-Ritz: RCF_RR_FP64 (cuBLAS), RCF_RR_DF, RCF_RR_TC or
    RCF_RR_MIXED."""
    _check(ctx, lib().rcf_set_rr_arith(ctx, int(kind)))


def rcf_inner(ctx, Y, Z, C, w=None, arith: int = 2, nrows=None):
    """C (nz, n) complex128 tensor receives Y^H diag(w) Z (C[j, i] = C(i, j): rows of the tensors are
    columns); Y (n, rows), Z (nz, rows) complex128; w a float64 CUDA tensor of rows / 2 node weights."""
    import torch
    py, ldy = _dev(Y, torch.complex128, "Y")
    pz, ldz = _dev(Z, torch.complex128, "Z")
    pc, ldc = _dev(C, torch.complex128, "C")
    rows = Y.shape[1] if nrows is None else int(nrows)
    if C.shape[0] < Z.shape[0] or C.shape[1] < Y.shape[0]:
        raise ValueError("C must be (nz, >= n)")
    pw = None
    if w is not None:
        if w.dtype != torch.float64 or not w.is_cuda:
            raise TypeError("w must be a float64 CUDA tensor")
        pw = ctypes.c_void_p(w.data_ptr())
    _check(ctx, lib().rcf_inner(ctx, py, ldy, Y.shape[0], pz, ldz, Z.shape[0], rows, pw, pc, ldc, int(arith)))


def rcf_rotate(ctx, Y, Q, X, arith: int = 2, nrows=None):
    """X (n, rows) complex128 receives Y Q for Y (n, rows) and Q (n, n) complex128 (Q[j, i] = Q(i, j));
    X may be Y for arith = RCF_RR_TC."""
    import torch
    py, ldy = _dev(Y, torch.complex128, "Y")
    pq, ldq = _dev(Q, torch.complex128, "Q")
    px, ldx = _dev(X, torch.complex128, "X")
    rows = Y.shape[1] if nrows is None else int(nrows)
    _check(ctx, lib().rcf_rotate(ctx, py, ldy, Y.shape[0], pq, ldq, rows, px, ldx, int(arith)))


def _field(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def rcf_op_set_gauss(ctx, op, nq: int) -> None:
    """Switch op to the full consistent mass with nq Gauss points per direction."""
    _check(ctx, lib().rcf_op_set_gauss(op, int(nq)))


def rcf_op_gauss_points(ctx, op, ncells: int, nq: int) -> np.ndarray:
    out = np.empty((ncells, nq ** 3, 3), dtype=np.float64)
    _check(ctx, lib().rcf_op_gauss_points(op, _np_ptr(out)))
    return out


def rcf_mass_apply(ctx, op, X, Y, prec: int = RCF_FP64):
    """Y = M X (complex tensors of shape (nvec, 2M))."""
    px, ldx = _dev_mv(X, prec, "X")
    py, ldy = _dev_mv(Y, prec, "Y")
    _check(ctx, lib().rcf_mass_apply(ctx, op, px, ldx, X.shape[0], py, ldy, int(prec)))


def rcf_workspace_bytes(ctx) -> int:
    """Bytes of device scratch memory the context holds."""
    return int(lib().rcf_workspace_bytes(ctx))


def rcf_laplacian(ctx, mesh, x, y):
    """y = K x (scalar nodal fields, float64 CUDA tensors of nnodes entries)."""
    _check(ctx, lib().rcf_laplacian(ctx, mesh, _field(x, "x"), _field(y, "y")))


def rcf_poisson_pcg(ctx, mesh, f, x, cheb_degree: int, a: float, b: float, tol: float, maxit: int):
    """Solve K x = f (x: initial guess in, solution out); returns (iterations, final ||r||)."""
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    _check(ctx, lib().rcf_poisson_pcg(ctx, mesh, _field(f, "f"), _field(x, "x"), int(cheb_degree), float(a),
                                      float(b), float(tol), int(maxit), ctypes.byref(it), ctypes.byref(res)))
    return it.value, res.value


def rcf_set_wait_limit(ctx, polls: int) -> None:
    _check(ctx, lib().rcf_set_wait_limit(ctx, int(polls)))


def rcf_set_step_kernel(ctx, kind: int) -> None:
    """FP32 step kernel of this context: RCF_STEP_CPASYNC (default) or RCF_STEP_TMA."""
    _check(ctx, lib().rcf_set_step_kernel(ctx, int(kind)))


def rcf_apply_noalloc(ctx, op, form: int, X, Y, prec: int = RCF_FP64):
    """rcf_apply that allocates nothing (fixed scratch inside the library; natoms * nvec <= 16384)."""
    import torch
    dt = torch.complex128 if prec == RCF_FP64 else torch.complex64
    px, ldx = _dev(X, dt, "X")
    py, ldy = _dev(Y, dt, "Y")
    nvec = X.shape[0] if X.dim() == 2 else 1
    _check(ctx, lib().rcf_apply_noalloc(ctx, op, form, px, ldx, nvec, py, ldy, prec))


# ---- block floating-point codec (Section III-C-3) ----------------------------------

RCF_BFP_RATES = (16, 12, 10)


def rcf_bfp_stream_bytes(n: int, nbits: int) -> int:
    """Bytes of the compressed stream of n FP32 values at nbits per value."""
    r = lib().rcf_bfp_stream_bytes(int(n), int(nbits))
    if r < 0:
        raise ValueError(f"invalid n={n} or nbits={nbits} (rates {RCF_BFP_RATES})")
    return int(r)


def _flat(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def rcf_bfp_encode(ctx, x, nbits: int, stream):
    """Encode the float32 CUDA tensor x (contiguous, any shape) into the uint8 CUDA tensor
    stream (at least rcf_bfp_stream_bytes(x.numel(), nbits) bytes)."""
    import torch
    px = _flat(x, torch.float32, "x")
    ps = _flat(stream, torch.uint8, "stream")
    if nbits in RCF_BFP_RATES and stream.numel() < rcf_bfp_stream_bytes(x.numel(), nbits):
        raise ValueError("stream is too small")
    _check(ctx, lib().rcf_bfp_encode(ctx, px, x.numel(), int(nbits), ps))


def rcf_bfp_decode(ctx, stream, nbits: int, y):
    """Decode y.numel() values from the uint8 CUDA tensor stream into the float32 CUDA
    tensor y (contiguous, any shape)."""
    import torch
    ps = _flat(stream, torch.uint8, "stream")
    py = _flat(y, torch.float32, "y")
    if nbits in RCF_BFP_RATES and stream.numel() < rcf_bfp_stream_bytes(y.numel(), nbits):
        raise ValueError("stream is too small")
    _check(ctx, lib().rcf_bfp_decode(ctx, ps, y.numel(), int(nbits), py))
