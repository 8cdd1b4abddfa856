"""Full consistent mass with Gauss-Legendre quadrature (Section III-A; Section III-B-2)
(TEST INFRASTRUCTURE ONLY).

The paper keeps the full FE mass M_{2I+a,2J+b} = delta_ab int N_I N_J for the
noncollinear problem and evaluates every cell integral with a Gauss-Legendre rule
of sufficient order; the filter then uses a diagonal D (GLL-integrated or lumped
mass) in place of M^-1, and R-ChFSI still converges to the eigenpairs of
H x = eps M x, whereas ChFSI with D in place of M stagnates (Section III-B-2,
text after Eq. ChFSIrecurrence and Eq. rChFSIrecurrence).

This module assembles, on the periodic GLL mesh of ``Mesh``:
- the tensor-product Lagrange basis (degree p on the GLL nodes) and its
  derivatives at the n_q^3 Gauss-Legendre points of a cell;
- per cell, by the definition of each integral as a quadrature sum,
  mass    M^e = N^T diag(w |J|) N,
  kinetic K^e = 1/2 sum_d G_d^T diag(w |J|) G_d,
  potential blocks V^e = N^T diag(w |J| V_q) N and B^e_d likewise, combined per
  spin pair as V delta_ab + sum_d B_d (sigma_d)_ab (Eq. hloc);
- spin-orbit projector columns p_I = int N_I beta over the cells (Eq. hnloc,
  with the same p-type Gaussians as ``Hamiltonian``);
- D = the GLL-integrated diagonal (``Mesh.lumped_mass``), used in place of M^-1.

The object exposes ``apply`` (H X), ``mass_apply`` (M X), ``mass_solve`` (M^-1 X,
sparse LU) and ``Mdiag`` (D, per spinor row), so the filters, the residual, the
Rayleigh-Ritz step and Algorithm 1 of this package run on it unchanged: the
residual and the Gram matrix use the full M, the filters use D.

Parity: pinned in tests/test_oracle_fullmass.py: the Lagrange tables against the
GLL derivative matrix and polynomial reproduction; M symmetric positive definite
with row sums equal to the GLL-integrated mass and independent of n_q >= p + 1;
the free-electron and harmonic-oscillator spectra equal sums of 1D generalized
eigenvalues whose 1D matrices come from exact polynomial integration; Galerkin
upper bounds of the plane-wave levels; Hermiticity and Kramers pairs; and the
paper's claim that R-ChFSI with D reaches the dense eigenvalues of (H, M) while
ChFSI with D stalls.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .hamiltonian import PAULI, soc_delta
from .mesh import Mesh


def lagrange_tables(xi: np.ndarray, x: np.ndarray):
    """Values B[q, a] = l_a(x_q) and derivatives Dq[q, a] = l_a'(x_q) of the Lagrange
    polynomials on the nodes xi, by the product formula and its derivative."""
    n = xi.size
    B = np.ones((x.size, n))
    Dq = np.zeros((x.size, n))
    for a in range(n):
        others = [b for b in range(n) if b != a]
        den = np.prod([xi[a] - xi[b] for b in others])
        B[:, a] = np.prod([x - xi[b] for b in others], axis=0) / den if others else 1.0
        for m in others:
            rest = [b for b in others if b != m]
            term = np.prod([x - xi[b] for b in rest], axis=0) if rest else np.ones_like(x)
            Dq[:, a] += term / den
    return B, Dq


class FullMassHamiltonian:
    """H and the full consistent M on ``mesh``, integrals by n_q-point Gauss-Legendre rules.

    Vq: (ncells, n_q^3) potential at the Gauss points of each cell (local point
    q = qx + n_q (qy + n_q qz)); Bq: (3, ncells, n_q^3) or None.
    """

    def __init__(self, mesh: Mesh, nq: int, Vq, Bq=None, atoms=None, proj_width=None, proj_h=None,
                 rcut_factor: float = 5.0):
        self.mesh = mesh
        self.nq = int(nq)
        M = mesh.nnodes
        self.nnodes, self.N = M, 2 * M
        g, wg = np.polynomial.legendre.leggauss(self.nq)
        self.gauss, self.gauss_w = g, wg
        B1, D1 = lagrange_tables(mesh.xi, g)
        # 3D tables: row q = qx + n_q (qy + n_q qz), column l = a + n_p (b + n_p c)
        self.Nq = np.kron(B1, np.kron(B1, B1))
        G = [(2.0 / mesh.h[0]) * np.kron(B1, np.kron(B1, D1)),
             (2.0 / mesh.h[1]) * np.kron(B1, np.kron(D1, B1)),
             (2.0 / mesh.h[2]) * np.kron(D1, np.kron(B1, B1))]
        self.wq = np.kron(wg, np.kron(wg, wg)) * mesh.detJ           # w_q |J|
        Wq = np.diag(self.wq)
        nloc = mesh.nloc
        Vq = np.asarray(Vq, dtype=np.float64).reshape(mesh.ncells, self.nq ** 3)
        Bq = (np.zeros((3, mesh.ncells, self.nq ** 3)) if Bq is None
              else np.asarray(Bq, dtype=np.float64).reshape(3, mesh.ncells, self.nq ** 3))
        self.Vq, self.Bq = Vq, Bq
        Me = self.Nq.T @ Wq @ self.Nq
        Ke = 0.5 * sum(Gd.T @ Wq @ Gd for Gd in G)
        self.Me, self.Ke = Me, Ke
        Ms = mesh.assemble(Me)
        Ks = mesh.assemble(Ke)
        # potential: one element matrix per cell and field component
        rows = np.repeat(mesh.conn, nloc, axis=1).ravel()
        cols = np.tile(mesh.conn, (1, nloc)).ravel()

        def assemble_field(F):
            blocks = np.einsum("ql,eq,qm->elm", self.Nq, F * self.wq[None, :], self.Nq)
            A = sp.coo_matrix((blocks.ravel(), (rows, cols)), shape=(M, M)).tocsr()
            A.sum_duplicates()
            return A

        Pv = assemble_field(Vq)
        Pb = [assemble_field(Bq[d]) for d in range(3)]
        I2 = sp.identity(2, format="csr")
        self.Mscalar = Ms
        self.M = sp.kron(Ms, I2, format="csr")
        Hloc = sp.kron(Ks + Pv, I2, format="csr").astype(np.complex128)
        for d in range(3):
            Hloc = Hloc + sp.kron(Pb[d], sp.csr_matrix(PAULI[d]), format="csr")
        self.Hloc = Hloc.tocsr()
        self.mass = mesh.lumped_mass()                 # D_I (GLL-integrated)
        self.Mdiag = np.repeat(self.mass, 2)
        self._lu = None
        self.projectors = []
        if atoms is not None and len(atoms) > 0:
            self._build_projectors(np.asarray(atoms, float), np.asarray(proj_width, float),
                                   np.asarray(proj_h, float), rcut_factor)

    def gauss_coords(self) -> np.ndarray:
        """Coordinates of the Gauss points per cell, shape (ncells, n_q^3, 3), in [0, L)."""
        mesh, nq = self.mesh, self.nq
        nx, ny, nz = (int(v) for v in mesh.n)
        ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        c, b, a = np.meshgrid(np.arange(nq), np.arange(nq), np.arange(nq), indexing="ij")
        out = np.empty((mesh.ncells, nq ** 3, 3))
        for d, (ecell, loc) in enumerate(((ex, a), (ey, b), (ez, c))):
            out[:, :, d] = (ecell.reshape(-1, 1) * mesh.h[d]
                            + (self.gauss[loc.reshape(1, -1)] + 1.0) * mesh.h[d] / 2.0)
        return out

    def _build_projectors(self, atoms, widths, hcoup, rcut_factor):
        mesh = self.mesh
        xq = self.gauss_coords()
        L = mesh.L
        for a in range(atoms.shape[0]):
            d = xq - atoms[a]
            d = d - L * np.round(d / L)                   # minimum image
            r2 = np.sum(d * d, axis=2)
            col = np.zeros((mesh.nnodes, 6))              # int N_I beta_{j,i}
            for j in range(2):
                s = widths[a, j]
                Nj = np.sqrt(2.0 / (np.pi ** 1.5 * s ** 5))
                gj = Nj * np.exp(-r2 / (2.0 * s * s)) * (r2 < (rcut_factor * s) ** 2)
                for i in range(3):
                    f = gj * d[:, :, i] * self.wq[None, :]            # (ncells, nq^3)
                    per_node = f @ self.Nq                             # (ncells, nloc)
                    col[:, 3 * j + i] = np.bincount(mesh.conn.ravel(), weights=per_node.ravel(),
                                                    minlength=mesh.nnodes)
            supp = np.nonzero(np.any(col != 0.0, axis=1))[0]
            P = np.zeros((2 * supp.size, 12))
            for j in range(2):
                for i in range(3):
                    for sg in range(2):
                        P[sg::2, 6 * j + 2 * i + sg] = col[supp, 3 * j + i]
            rows = np.empty(2 * supp.size, dtype=np.int64)
            rows[0::2] = 2 * supp
            rows[1::2] = 2 * supp + 1
            self.projectors.append(dict(support=supp, rows=rows, P=P,
                                        Delta=soc_delta(hcoup[a, 0], hcoup[a, 1]), h=hcoup[a].copy()))

    # -- actions ----------------------------------------------------------
    def apply(self, X: np.ndarray) -> np.ndarray:
        """H X for X of shape (2M, nvec) (or (2M,))."""
        Y = self.Hloc @ X
        for pr in self.projectors:
            C = pr["P"].T @ X[pr["rows"]]
            Y[pr["rows"]] += pr["P"] @ (pr["Delta"] @ C)
        return Y

    def mass_apply(self, X: np.ndarray) -> np.ndarray:
        """M X with the full consistent mass."""
        return self.M @ X

    def mass_solve(self, X: np.ndarray) -> np.ndarray:
        """M^-1 X (sparse LU of the scalar mass, applied per spin component)."""
        if self._lu is None:
            self._lu = spla.splu(self.Mscalar.tocsc())
        X = np.asarray(X)
        out = np.empty_like(X, dtype=np.result_type(X.dtype, np.float64))
        for s in range(2):
            b = X[s::2]
            if np.iscomplexobj(b):
                out[s::2] = (self._lu.solve(np.ascontiguousarray(b.real))
                             + 1j * self._lu.solve(np.ascontiguousarray(b.imag)))
            else:
                out[s::2] = self._lu.solve(np.ascontiguousarray(b))
        return out

    def dense(self):
        """Dense (H, M) for brute-force checks on tiny meshes."""
        H = self.Hloc.toarray()
        for pr in self.projectors:
            r = pr["rows"]
            H[np.ix_(r, r)] += pr["P"] @ pr["Delta"] @ pr["P"].T
        return H, self.M.toarray()
