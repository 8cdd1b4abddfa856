"""torch.autograd wrappers around the filter and its adjoint.

``RChFSIFilter`` maps the quadrature-point fields V, B and the spin-orbit
couplings h to the filtered block Y_q (X, Lambda and the bounds held fixed);
its backward is one ``rcf_adjoint_filter`` call (the reverse recurrence with
checkpoints, all in the library's kernels).  ``RitzValues`` maps a block Y (and
the operator) to its Rayleigh-Ritz values; its backward gives
dtheta_j = 2 Re x_j^H (H - theta_j M) dY q_j + x_j^H dH x_j, with x_j = Y q_j the
M-normalised Ritz vectors, all of it in one ``rcf_ritz_cotangent`` call.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rchfsi as R


class Operator:
    """Context + mesh + operator whose V, B, h are torch tensors (FP64)."""

    def __init__(self, problem):
        self.p = problem
        self.ctx, self.op, self.mesh = problem.ctx, problem.op, problem.mesh
        self.natoms = problem.natoms
        self.mass = torch.from_numpy(R.rcf_mesh_mass(self.mesh)).cuda()
        self.mdiag = self.mass.repeat_interleave(2)
        self._state = None

    def set(self, V: torch.Tensor, B: torch.Tensor, h: torch.Tensor):
        key = (V.data_ptr(), V._version, B.data_ptr(), B._version, h.data_ptr(), h._version)
        if key == self._state:
            return
        R.rcf_potential_set(self.ctx, self.op, V.detach().contiguous(), B.detach().contiguous())
        if self.natoms:
            R.rcf_projectors_couplings(self.ctx, self.op, h.detach().cpu().numpy())
        self._state = key


class RChFSIFilter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, B, h, opw: Operator, X, ritz, bounds, degree: int, prec: int, ckpt: int):
        opw.set(V, B, h)
        Y = torch.empty_like(X)
        R.rcf_filter(opw.ctx, opw.op, X, ritz, degree, bounds, R.RCF_RCHFSI, prec, 0, Y)
        ctx.opw, ctx.X, ctx.ritz, ctx.bounds = opw, X, ritz, bounds
        ctx.degree, ctx.prec, ctx.ckpt = degree, prec, ckpt
        ctx.shapes = (V.shape, B.shape, h.shape)
        ctx.save_for_backward(V, B, h)
        return Y

    @staticmethod
    def backward(ctx, Ybar):
        V, B, h = ctx.saved_tensors
        opw = ctx.opw
        opw.set(V, B, h)
        dV = torch.zeros_like(V)
        dB = torch.zeros_like(B)
        dh = np.zeros((max(opw.natoms, 1), 2))
        R.rcf_adjoint_filter(opw.ctx, opw.op, ctx.X, ctx.ritz, ctx.degree, ctx.bounds, R.RCF_RCHFSI,
                             ctx.prec, Ybar.contiguous(), ctx.ckpt, dV, dB,
                             dh if opw.natoms else None)
        dht = torch.from_numpy(dh[:opw.natoms]).to(h.device, h.dtype) if opw.natoms else torch.zeros_like(h)
        return dV, dB, dht, None, None, None, None, None, None, None


class RitzValues(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y, V, B, h, opw: Operator):
        opw.set(V, B, h)
        Yw = Y.detach().clone()
        Xr = torch.empty_like(Yw)
        theta = R.rcf_rayleigh_ritz(opw.ctx, opw.op, Yw, Xr)
        th = torch.from_numpy(theta).to(Y.device)
        ctx.opw = opw
        ctx.save_for_backward(Y, Xr, th, V, B, h)
        return th

    @staticmethod
    def backward(ctx, thbar):
        Y, Xr, th, V, B, h = ctx.saved_tensors
        opw = ctx.opw
        opw.set(V, B, h)
        Ybar = torch.empty_like(Y)
        dV = torch.zeros_like(V)
        dB = torch.zeros_like(B)
        dh = np.zeros((max(opw.natoms, 1), 2))
        R.rcf_ritz_cotangent(opw.ctx, opw.op, Y.detach().contiguous(), Xr, th.cpu().numpy(),
                             thbar.detach().cpu().numpy(), Ybar, dV, dB, dh if opw.natoms else None)
        dht = torch.from_numpy(dh[:opw.natoms]).to(h.device, h.dtype) if opw.natoms else torch.zeros_like(h)
        return Ybar, dV, dB, dht, None
