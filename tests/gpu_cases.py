"""Helpers shared by the GPU parity tests (test helper, not a test module)."""
import dataclasses

import numpy as np

import workloads
from oracle_cases import build_oracle


def torch():
    import torch as _t
    return _t


def to_dev(X, dtype=None):
    t = torch()
    X = np.asarray(X)
    if X.ndim == 1:
        X = X[:, None]
    d = t.from_numpy(np.ascontiguousarray(X.T)).to("cuda")
    return d if dtype is None else d.to(dtype)


def to_host(T):
    return T.detach().to("cpu").numpy().T.astype(np.complex128)


def mesh_workload(ncell, side, p, natoms=2, seed=11, bmax=0.05):
    base = workloads.workload("cfg1")
    return dataclasses.replace(base, name="case", ncell=ncell, side=side, p=p, natoms=natoms,
                               lattice=None, ngauss=4, bmax=bmax, seed=seed)


class Pair:
    """The same synthetic problem on the oracle and on the GPU (identical V, B, projector inputs)."""

    def __init__(self, ncell, side, p, natoms=2, seed=11, assemble=True, with_b=True, with_proj=True):
        from paper_2605_30128_gb300.problem import GPUProblem
        from oracle import Hamiltonian, Mesh
        self.w = mesh_workload(ncell, side, p, natoms=natoms, seed=seed)
        prm = workloads.draw_parameters(self.w)
        self.params = prm
        mesh = Mesh(ncell, side, p)
        q = mesh.quad_coords().reshape(-1, 3)
        V = workloads.gaussian_sum_potential(q, prm["centres"], prm["depths"], prm["widths"], prm["L"])
        B = (workloads.smooth_periodic_field(q, prm["kvec"], prm["amps"], prm["phases"], prm["L"], prm["bmax"])
             if with_b else np.zeros((3, q.shape[0])))
        self.V = V.reshape(mesh.ncells, mesh.nloc)
        self.B = B.reshape(3, mesh.ncells, mesh.nloc)
        self.H = Hamiltonian(mesh, self.V, self.B, prm["atoms"] if with_proj else None,
                             prm["proj_width"], prm["proj_h"], assemble=assemble)
        self.g = GPUProblem(self.w, params=prm, with_b=with_b, with_proj=with_proj)
        self.g.set_potential(self.V, self.B)
        self.N = self.H.N

    def close(self):
        self.g.close()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
