"""Periodic hexahedral spectral-element mesh (Section III-A, Eq. FEWfns; Section III-B-2).

Uniform periodic box of n_x x n_y x n_z cells, Lagrange degree p on GLL
nodes, GLL quadrature collocated with the nodes, so the mass matrix is the
GLL-integrated (lumped) diagonal D = M that the filter uses (Section
III-B-2, text after Eq. ChFSIrecurrence).

Numbering (shared convention with the GPU library, each side implementing
it independently):
  global node  I = i + G_x (j + G_y k),  G_d = n_d p, (i, j, k) node indices
  cell         e = e_x + n_x (e_y + n_y e_z)
  local node   l = a + n_p (b + n_p c),  n_p = p + 1
  conn[e, l]   = global node at ((e_x p + a) mod G_x, (e_y p + b) mod G_y, (e_z p + c) mod G_z)
  spinor row   2 I + alpha  (Section III-A: M_{2I+alpha, 2J+beta})

Parity: connectivity pinned by coordinate matching; element matrix pinned by
the free-electron tensor-product closed form (tests/test_oracle_fem.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .gll import gll_nodes_weights, lagrange_derivative_matrix


class Mesh:
    def __init__(self, ncell, side, p: int):
        self.n = np.array(np.broadcast_to(np.asarray(ncell, dtype=np.int64), (3,)))
        self.L = np.array(np.broadcast_to(np.asarray(side, dtype=np.float64), (3,)))
        if np.any(self.n < 1):
            raise ValueError("need at least one cell per direction")
        self.p = int(p)
        self.n_p = self.p + 1
        self.h = self.L / self.n
        self.G = self.n * self.p
        self.nnodes = int(np.prod(self.G))
        self.ncells = int(np.prod(self.n))
        self.nloc = self.n_p ** 3
        self.xi, self.w = gll_nodes_weights(self.p)
        self.D = lagrange_derivative_matrix(self.xi)
        self.detJ = float(np.prod(self.h)) / 8.0
        self.conn = self._connectivity()

    # -- numbering -------------------------------------------------------
    def _connectivity(self) -> np.ndarray:
        p, n_p = self.p, self.n_p
        nx, ny, nz = (int(v) for v in self.n)
        Gx, Gy, Gz = (int(v) for v in self.G)
        # cell indices (e_z, e_y, e_x) and local indices (c, b, a), slowest first
        ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        c, b, a = np.meshgrid(np.arange(n_p), np.arange(n_p), np.arange(n_p), indexing="ij")
        i = (ex.reshape(-1, 1) * p + a.reshape(1, -1)) % Gx
        j = (ey.reshape(-1, 1) * p + b.reshape(1, -1)) % Gy
        k = (ez.reshape(-1, 1) * p + c.reshape(1, -1)) % Gz
        return (i + Gx * (j + Gy * k)).astype(np.int64)

    def node_coords(self) -> np.ndarray:
        """Coordinates of global nodes in [0, L), shape (nnodes, 3)."""
        out = []
        for d in range(3):
            idx = np.arange(self.G[d])
            out.append((idx // self.p) * self.h[d] + (self.xi[idx % self.p] + 1.0) * self.h[d] / 2.0)
        X, Y, Z = np.meshgrid(out[0], out[1], out[2], indexing="ij")
        # global index i + Gx (j + Gy k): i fastest
        return np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                         Z.transpose(2, 1, 0).ravel()], axis=1)

    def quad_coords(self) -> np.ndarray:
        """Quadrature-point (= local GLL node) coordinates per cell, shape (ncells, n_p^3, 3), unwrapped."""
        n_p = self.n_p
        nx, ny, nz = (int(v) for v in self.n)
        ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        c, b, a = np.meshgrid(np.arange(n_p), np.arange(n_p), np.arange(n_p), indexing="ij")
        out = np.empty((self.ncells, self.nloc, 3))
        for d, (ecell, loc) in enumerate(((ex, a), (ey, b), (ez, c))):
            out[:, :, d] = (ecell.reshape(-1, 1) * self.h[d]
                            + (self.xi[loc.reshape(1, -1)] + 1.0) * self.h[d] / 2.0)
        return out

    def quad_weights(self) -> np.ndarray:
        """w_q |J| for the local points l = a + n_p (b + n_p c), shape (n_p^3,)."""
        w = self.w
        return np.kron(w, np.kron(w, w)) * self.detJ

    # -- element and global matrices --------------------------------------
    def element_kinetic(self) -> np.ndarray:
        """K^e_IJ = 1/2 int grad N_I . grad N_J over one cell, by GLL quadrature.

        Gradients of the tensor-product basis at the GLL points: the basis
        factor in the differentiated direction gives D (times 2/h_d), the
        other two factors are Kronecker deltas (Section III-A; the Laplacian
        term of Eq. hloc, -1/2 nabla^2).
        """
        I = np.eye(self.n_p)
        Gx = (2.0 / self.h[0]) * np.kron(I, np.kron(I, self.D))
        Gy = (2.0 / self.h[1]) * np.kron(I, np.kron(self.D, I))
        Gz = (2.0 / self.h[2]) * np.kron(self.D, np.kron(I, I))
        Wq = np.diag(self.quad_weights())
        return 0.5 * (Gx.T @ Wq @ Gx + Gy.T @ Wq @ Gy + Gz.T @ Wq @ Gz)

    def lumped_mass(self) -> np.ndarray:
        """M_I = sum over cells and local points mapped to I of w_q |J| (GLL-integrated mass)."""
        wq = self.quad_weights()
        return np.bincount(self.conn.ravel(), weights=np.tile(wq, self.ncells), minlength=self.nnodes)

    def assemble(self, Ke: np.ndarray) -> sp.csr_matrix:
        """Global sum_e R_e^T K^e R_e as a scalar (nnodes x nnodes) CSR matrix."""
        Ii, Jj = np.nonzero(Ke)
        rows = self.conn[:, Ii].ravel()
        cols = self.conn[:, Jj].ravel()
        vals = np.tile(Ke[Ii, Jj], self.ncells)
        A = sp.coo_matrix((vals, (rows, cols)), shape=(self.nnodes, self.nnodes)).tocsr()
        A.sum_duplicates()
        return A

    def kinetic(self) -> sp.csr_matrix:
        return self.assemble(self.element_kinetic())

    # -- 1D factors (used only by closed-form tests) -----------------------
    def assembled_1d(self, d: int):
        """Periodic 1D stiffness K1g (with 2/h) and mass Wg (with h/2) along direction d."""
        p, G, h = self.p, int(self.G[d]), self.h[d]
        K1 = self.D.T @ np.diag(self.w) @ self.D
        K = np.zeros((G, G))
        W = np.zeros(G)
        for e in range(int(self.n[d])):
            idx = [(e * p + a) % G for a in range(self.n_p)]
            for a in range(self.n_p):
                W[idx[a]] += self.w[a] * h / 2.0
                for b in range(self.n_p):
                    K[idx[a], idx[b]] += K1[a, b] * 2.0 / h
        return K, W
