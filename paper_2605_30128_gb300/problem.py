"""Set up a synthetic workload on the GPU through the C ABI.

The mesh, quadrature points, potential blocks and projectors are all built by
librchfsi; this module only draws the workload's seeded parameters
(``workloads``) and evaluates the synthetic fields at the quadrature points
that the library reports.
"""
from __future__ import annotations

import numpy as np

import workloads
from . import rchfsi as R


class GPUProblem:
    """Context + mesh + operator for one workload (V, B and projectors set)."""

    def __init__(self, w: workloads.Workload, device: int = 0, stream=None, with_b: bool = True,
                 with_proj: bool = True, params: dict | None = None, ctx=None):
        self.w = w
        self.params = workloads.draw_parameters(w) if params is None else params
        self.own_ctx = ctx is None
        self.ctx = R.rcf_create(device, stream) if ctx is None else ctx
        self.mesh = R.rcf_mesh_create(self.ctx, w.ncell, w.side, w.p)
        self.nnodes, self.ncells, self.nloc = R.rcf_mesh_info(self.mesh)
        self.N = 2 * self.nnodes
        self.op = R.rcf_op_create(self.ctx, self.mesh)
        prm = self.params
        q = R.rcf_mesh_quadrature_points(self.mesh).reshape(-1, 3)
        V = workloads.gaussian_sum_potential(q, prm["centres"], prm["depths"], prm["widths"], prm["L"])
        B = (workloads.smooth_periodic_field(q, prm["kvec"], prm["amps"], prm["phases"], prm["L"], prm["bmax"])
             if with_b else np.zeros((3, q.shape[0])))
        self.V = V.reshape(self.ncells, self.nloc)
        self.B = B.reshape(3, self.ncells, self.nloc)
        R.rcf_potential_set(self.ctx, self.op, self.V, self.B)
        self.natoms = 0
        if with_proj and w.natoms > 0:
            R.rcf_projectors_set(self.ctx, self.op, prm["atoms"], prm["proj_width"], prm["proj_h"])
            self.natoms = w.natoms

    def set_potential(self, V, B):
        R.rcf_potential_set(self.ctx, self.op, V, B)

    def close(self):
        if self.op is not None:
            R.rcf_op_destroy(self.op)
            R.rcf_mesh_destroy(self.mesh)
            if self.own_ctx:
                R.rcf_destroy(self.ctx)
            self.op = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
