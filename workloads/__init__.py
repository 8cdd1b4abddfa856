"""Seeded synthetic inputs shared by the oracle and the GPU path.

This module holds no arithmetic of the method (no mesh, no quadrature, no
operator, no filter).  It only draws random parameters from a seed and
evaluates the synthetic fields (a Gaussian-sum potential, a smooth periodic
magnetic field) at coordinates that the caller supplies.  The oracle and the
GPU path each compute their own quadrature-point coordinates; both then feed
those coordinates through the same field formulas here.

Workloads stand in for the paper's twisted-bilayer systems (Section IV-B),
whose structures, pseudopotentials and meshes are not available: periodic
cubes meshed with hexahedral cells of edge 2 bohr (the paper's MoSe2 mesh is
2.1 bohr near nuclei), a local potential that is a sum of attractive
Gaussians, a smooth exchange-correlation-like field B, and atoms carrying
l = 1 spin-orbit projectors (Section II-A, Eq. hnloc).
"""
from __future__ import annotations

import dataclasses
from typing import Tuple

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "workload",
    "draw_parameters",
    "gaussian_sum_potential",
    "smooth_periodic_field",
    "complex_normal",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic problem: mesh, fields, atoms, block and filter sizes."""

    name: str
    ncell: int          # cells per direction (periodic cube)
    side: float         # cube side in bohr
    p: int              # Lagrange degree on GLL nodes
    natoms: int
    lattice: Tuple[int, int, int] | None  # jittered atom lattice, or None = uniform draw
    ngauss: int         # Gaussians in V (one per atom when lattice is set)
    bmax: float         # max |B| over quadrature points (Ha)
    nvec: int           # spinor vectors
    block: int          # band block size for the filter
    degree: int         # Chebyshev degree q
    cycles: int         # filter + Rayleigh-Ritz cycles
    lanczos: int        # Lanczos steps for the upper bound
    ckpt: int           # adjoint checkpoint interval
    seed: int

    @property
    def nodes_per_dir(self) -> int:
        return self.ncell * self.p

    @property
    def nnodes(self) -> int:
        return self.nodes_per_dir ** 3

    @property
    def ndof(self) -> int:
        """Complex spinor degrees of freedom (both components)."""
        return 2 * self.nnodes

    @property
    def ncells(self) -> int:
        return self.ncell ** 3


WORKLOADS = {
    # 4^3 cells, side 8, p=4: 8,192 complex DoF; 32 vectors, degree 10, 3 cycles.
    "cfg1": Workload("cfg1", 4, 8.0, 4, 2, None, 4, 0.05, 32, 32, 10, 3, 10, 5, 1001),
    # 16^3 cells, side 32, p=6: 1,769,472 DoF; 512 vectors, degree 30.
    "cfg2": Workload("cfg2", 16, 32.0, 6, 16, (2, 2, 4), 16, 0.10, 512, 512, 30, 1, 10, 5, 1002),
    # 20^3 cells, side 40, p=5: 2,000,000 DoF; 1024 vectors in blocks of 256, degree 40.
    "cfg3": Workload("cfg3", 20, 40.0, 5, 32, (2, 4, 4), 32, 0.10, 1024, 256, 40, 1, 10, 5, 1003),
    # 8^3 cells, side 16, p=4: 65,536 DoF; 64 vectors, degree 15, checkpoint every 5.
    "cfg4": Workload("cfg4", 8, 16.0, 4, 4, (2, 2, 1), 4, 0.10, 64, 64, 15, 1, 10, 5, 1004),
    # 20^3 cells, side 40, p=6: 3,456,000 DoF; 1024 vectors in blocks of 256, degree 50, 5 cycles.
    "cfg5": Workload("cfg5", 20, 40.0, 6, 64, (4, 4, 4), 64, 0.10, 1024, 256, 50, 5, 10, 5, 1005),
}


def workload(name: str, **overrides) -> Workload:
    """Return a named workload, optionally with fields replaced (e.g. a smaller nvec)."""
    w = WORKLOADS[name]
    return dataclasses.replace(w, **overrides) if overrides else w


def _minimum_image(d: np.ndarray, side: np.ndarray) -> np.ndarray:
    return d - side * np.round(d / side)


def draw_parameters(w: Workload) -> dict:
    """All random parameters of a workload, drawn from numpy PCG64(seed).

    Returns plain arrays: Gaussian centres/depths/widths, B wave vectors,
    amplitudes and phases, atom positions, projector widths and couplings.
    """
    rng = np.random.Generator(np.random.PCG64(w.seed))
    L = np.full(3, w.side)
    # atoms
    if w.lattice is None:
        atoms = rng.uniform(0.0, 1.0, size=(w.natoms, 3)) * L
    else:
        nx, ny, nz = w.lattice
        a = L / np.array([nx, ny, nz], dtype=float)
        grid = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
        base = (grid + 0.5) * a
        jitter = rng.uniform(-0.1, 0.1, size=base.shape) * a
        atoms = base + jitter
        assert atoms.shape[0] == w.natoms
    # Gaussian-sum local potential: seeded centres when the atoms are few,
    # otherwise one Gaussian per atom centred on it.
    if w.lattice is None:
        centres = rng.uniform(0.0, 1.0, size=(w.ngauss, 3)) * L
    else:
        centres = atoms.copy()
    depths = rng.uniform(1.0, 3.0, size=w.ngauss)
    widths = rng.uniform(0.8, 1.5, size=w.ngauss)
    # smooth periodic B: 4 plane waves per component with integer wave vectors
    kvec = rng.integers(-2, 3, size=(4, 3))
    kvec[np.all(kvec == 0, axis=1)] = np.array([1, 0, 0])
    amps = rng.normal(size=(3, 4))
    phases = rng.uniform(0.0, 2.0 * np.pi, size=(3, 4))
    # spin-orbit projectors: widths per channel j in {1/2, 3/2} and couplings (Ha)
    proj_width = rng.uniform(0.6, 0.75, size=(w.natoms, 2))
    proj_h = rng.uniform(0.01, 0.1, size=(w.natoms, 2))
    return dict(L=L, centres=centres, depths=depths, widths=widths, kvec=kvec, amps=amps,
                phases=phases, atoms=atoms, proj_width=proj_width, proj_h=proj_h, bmax=w.bmax)


def gaussian_sum_potential(coords: np.ndarray, centres: np.ndarray, depths: np.ndarray,
                           widths: np.ndarray, L: np.ndarray) -> np.ndarray:
    """V(r) = -sum_i d_i exp(-|r - c_i|^2 / (2 w_i^2)), minimum-image distance in the periodic box."""
    coords = np.asarray(coords, dtype=np.float64).reshape(-1, 3)
    V = np.zeros(coords.shape[0])
    for c, d, s in zip(centres, depths, widths):
        r = _minimum_image(coords - c, L)
        V -= d * np.exp(-np.sum(r * r, axis=1) / (2.0 * s * s))
    return V


def smooth_periodic_field(coords: np.ndarray, kvec: np.ndarray, amps: np.ndarray, phases: np.ndarray,
                          L: np.ndarray, bmax: float) -> np.ndarray:
    """B_d(r) = s * sum_m a_dm cos(2 pi k_m . r / L + phi_dm), d = x, y, z.

    The scale s makes max_r |B(r)| over the given coordinates equal to bmax.
    Returns an array of shape (3, npoints).
    """
    coords = np.asarray(coords, dtype=np.float64).reshape(-1, 3)
    arg = 2.0 * np.pi * (coords / L) @ kvec.T            # (npts, 4)
    B = np.empty((3, coords.shape[0]))
    for d in range(3):
        B[d] = np.cos(arg + phases[d][None, :]) @ amps[d]
    mag = np.sqrt(np.sum(B * B, axis=0)).max()
    return B * (bmax / mag) if mag > 0 else B


def complex_normal(seed: int, shape, dtype=np.complex128) -> np.ndarray:
    """(a + i b)/sqrt(2) with a, b ~ N(0, 1) from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.normal(size=shape)
    b = rng.normal(size=shape)
    return ((a + 1j * b) / np.sqrt(2.0)).astype(dtype)


def bfp_values(seed: int, n: int) -> np.ndarray:
    """float32[n] for the block floating-point codec, from PCG64(seed): each group of four
    consecutive values shares a scale drawn log-uniformly over the whole FP32 range
    (2^-149 .. 2^127), and each value a further factor 2^-u, u ~ U(0, 24), and a random
    sign; one group in 64 is all zero.  Residual blocks behave like this: neighbouring
    entries have similar magnitudes and the magnitudes span many decades."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = (n + 3) // 4
    scale = 2.0 ** rng.uniform(-149.0, 127.0, size=(g, 1))
    spread = 2.0 ** -rng.uniform(0.0, 24.0, size=(g, 4))
    sign = rng.choice([-1.0, 1.0], size=(g, 4))
    x = scale * spread * sign
    x[rng.random(g) < 1.0 / 64.0] = 0.0
    return x.astype(np.float32).ravel()[:n]
