"""Small problem builders for the oracle tests (test helper, not a test module)."""
import dataclasses

import numpy as np

import workloads
from oracle import Hamiltonian, Mesh


def small_workload(ncell=2, side=6.0, p=3, natoms=2, bmax=0.05, seed=7, **kw):
    base = workloads.workload("cfg1")
    return dataclasses.replace(base, name="small", ncell=ncell, side=side, p=p, natoms=natoms,
                               lattice=None, ngauss=4, bmax=bmax, seed=seed, **kw)


def build_oracle(w, with_b=True, with_proj=True, params=None):
    """Oracle Hamiltonian for a workload (V, B evaluated at the oracle's quadrature points)."""
    prm = workloads.draw_parameters(w) if params is None else params
    mesh = Mesh(w.ncell, w.side, w.p)
    q = mesh.quad_coords().reshape(-1, 3)
    V = workloads.gaussian_sum_potential(q, prm["centres"], prm["depths"], prm["widths"], prm["L"])
    B = (workloads.smooth_periodic_field(q, prm["kvec"], prm["amps"], prm["phases"], prm["L"], prm["bmax"])
         if with_b else np.zeros((3, q.shape[0])))
    H = Hamiltonian(mesh, V.reshape(mesh.ncells, mesh.nloc), B.reshape(3, mesh.ncells, mesh.nloc),
                    prm["atoms"] if with_proj else None, prm["proj_width"], prm["proj_h"])
    return H, prm, V.reshape(mesh.ncells, mesh.nloc), B.reshape(3, mesh.ncells, mesh.nloc)
