"""Discrete NC-SOC Hamiltonian H = H_loc + H_nloc and lumped mass M (Sections II-A, III-A).

H_loc (Eq. hloc): kinetic -1/2 nabla^2 times the 2x2 identity, plus the
spinor potential V I + B . sigma, integrated with GLL quadrature at the
nodes.  With the spinor row 2I + alpha (Section III-A) the potential adds the
2x2 block sum_e w_q |J| (V_q^e I + B_q^e . sigma) to node I's diagonal block
(the cell-level structure of Eq. cellHam).

H_nloc (Eq. hnloc, Section III-B-3 stage iv): separable, per atom a,
H_nloc = sum_a P_a Delta_a P_a^H with P_a the (2M x 12) cell-assembled
projector matrix and Delta_a a 12 x 12 Hermitian spin-orbit coupling matrix.
The paper does not give the projector form; the reading used here is three
real p-type Gaussians per channel j in {1/2, 3/2},
beta_{j,i}(r) = N_j d_i exp(-|d|^2 / (2 s_j^2)) (d the minimum-image offset,
cut at |d| < 5 s_j, int beta^2 = 1), and Delta_a = h_{1/2} P_{1/2} (+)
h_{3/2} P_{3/2} with the l = 1 spin-orbit projectors
P_{3/2} = (2 + L.sigma)/3, P_{1/2} = (1 - L.sigma)/3 on the (p orbital x
spin) space, (L_k)_{ij} = -i eps_{kij}.  The projector column (j, i, sigma)
holds M_I beta_{j,i}(x_I) in row 2I + sigma (GLL quadrature of
int N_I beta).

Parity: pinned by Hermiticity, Kramers degeneracy, spin-rotation invariance
with SOC off, the free-electron and harmonic-oscillator closed forms, and
dense brute force (tests/test_oracle_physics.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Mesh

PAULI = np.array([
    [[0, 1], [1, 0]],
    [[0, -1j], [1j, 0]],
    [[1, 0], [0, -1]],
], dtype=np.complex128)


def p_orbital_L() -> np.ndarray:
    """(L_k)_{ij} = -i eps_{kij} on the real p orbitals (x, y, z); shape (3, 3, 3)."""
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    return -1j * eps


def soc_delta(h_half: float, h_three_half: float) -> np.ndarray:
    """12 x 12 coupling matrix, index f = 6 j + 2 i + sigma (j: 0 -> 1/2, 1 -> 3/2)."""
    L = p_orbital_L()
    Ls = sum(np.kron(L[k], PAULI[k]) for k in range(3))
    I6 = np.eye(6)
    P_half = (I6 - Ls) / 3.0
    P_3half = (2.0 * I6 + Ls) / 3.0
    Delta = np.zeros((12, 12), dtype=np.complex128)
    Delta[:6, :6] = h_half * P_half
    Delta[6:, 6:] = h_three_half * P_3half
    return Delta


def channel_projector(j: int) -> np.ndarray:
    """The 12 x 12 derivative d Delta / d h_j (P_j placed in block j)."""
    e = np.zeros(2)
    e[j] = 1.0
    return soc_delta(e[0], e[1])


class Hamiltonian:
    """Sparse local part + low-rank nonlocal part; all FP64."""

    def __init__(self, mesh: Mesh, Vq: np.ndarray, Bq: np.ndarray | None = None,
                 atoms: np.ndarray | None = None, proj_width: np.ndarray | None = None,
                 proj_h: np.ndarray | None = None, rcut_factor: float = 5.0, assemble: bool = True):
        self.mesh = mesh
        M = mesh.nnodes
        self.nnodes = M
        self.N = 2 * M
        Vq = np.asarray(Vq, dtype=np.float64).reshape(mesh.ncells, mesh.nloc)
        Bq = (np.zeros((3, mesh.ncells, mesh.nloc)) if Bq is None
              else np.asarray(Bq, dtype=np.float64).reshape(3, mesh.ncells, mesh.nloc))
        self.Vq, self.Bq = Vq, Bq
        self.mass = mesh.lumped_mass()                # M_I
        self.Mdiag = np.repeat(self.mass, 2)          # row 2I + alpha
        # potential: per node 2x2 block sum_e w_q |J| (V I + B . sigma)
        wq = np.tile(mesh.quad_weights(), mesh.ncells)
        cidx = mesh.conn.ravel()
        pv = np.bincount(cidx, weights=wq * Vq.ravel(), minlength=M)
        pb = [np.bincount(cidx, weights=wq * Bq[d].ravel(), minlength=M) for d in range(3)]
        self.pv, self.pb = pv, pb
        self.projectors = []
        if atoms is not None and len(atoms) > 0:
            self._build_projectors(np.asarray(atoms, float), np.asarray(proj_width, float),
                                   np.asarray(proj_h, float), rcut_factor)
        self.Hloc = None
        if not assemble:
            return
        # kinetic, spin-diagonal
        K = mesh.kinetic()
        Hk = sp.kron(K, sp.identity(2, format="csr"), format="csr").astype(np.complex128)
        rows, cols, vals = [], [], []
        I = np.arange(M)
        for al in range(2):
            for be in range(2):
                v = pv * (1.0 if al == be else 0.0) + sum(pb[d] * PAULI[d][al, be] for d in range(3))
                rows.append(2 * I + al)
                cols.append(2 * I + be)
                vals.append(v)
        Hp = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(self.N, self.N)).tocsr()
        self.Hloc = (Hk + Hp).tocsr()

    def _build_projectors(self, atoms, widths, hcoup, rcut_factor):
        mesh = self.mesh
        xyz = mesh.node_coords()
        L = mesh.L
        for a in range(atoms.shape[0]):
            d = xyz - atoms[a]
            d = d - L * np.round(d / L)                   # minimum image
            r2 = np.sum(d * d, axis=1)
            rc = rcut_factor * widths[a].max()
            supp = np.nonzero(r2 < rc * rc)[0]            # sorted node indices
            beta = np.zeros((supp.size, 6))               # column 3 j + i
            for j in range(2):
                s = widths[a, j]
                Nj = np.sqrt(2.0 / (np.pi ** 1.5 * s ** 5))
                g = Nj * np.exp(-r2[supp] / (2.0 * s * s)) * (r2[supp] < (rcut_factor * s) ** 2)
                for i in range(3):
                    beta[:, 3 * j + i] = g * d[supp, i]
            # P restricted to rows {2I, 2I+1 : I in supp}: column f = 6 j + 2 i + sigma
            P = np.zeros((2 * supp.size, 12))
            for j in range(2):
                for i in range(3):
                    for sg in range(2):
                        P[sg::2, 6 * j + 2 * i + sg] = self.mass[supp] * beta[:, 3 * j + i]
            rows = np.empty(2 * supp.size, dtype=np.int64)
            rows[0::2] = 2 * supp
            rows[1::2] = 2 * supp + 1
            self.projectors.append(dict(support=supp, rows=rows, beta=beta, P=P,
                                        Delta=soc_delta(hcoup[a, 0], hcoup[a, 1]), h=hcoup[a].copy()))

    # -- actions ----------------------------------------------------------
    def apply(self, X: np.ndarray) -> np.ndarray:
        """H X for X of shape (2M, nvec) (or (2M,))."""
        Y = self.Hloc @ X
        for pr in self.projectors:
            C = pr["P"].T @ X[pr["rows"]]                 # P^H X (P real)
            Y[pr["rows"]] += pr["P"] @ (pr["Delta"] @ C)
        return Y

    def apply_rows(self, X: np.ndarray, nodes, magnitudes: bool = False) -> np.ndarray:
        """Rows {2I, 2I+1 : I in nodes} of H X, each computed from the element matrices of the
        cells that contain I (no global assembly); shape (2 len(nodes), nvec).

        magnitudes=True returns instead the same sums taken over the moduli of every factor
        (|K^e| |X|, |potential block| |X|, |P| |Delta| |P^T| |X|): an upper bound of the sum
        of the magnitudes of the terms of each entry, the scale of its rounding error."""
        mesh = self.mesh
        Ke = mesh.element_kinetic()
        X = np.asarray(X).reshape(self.N, -1)
        if magnitudes:
            X = np.abs(X)
            Ke = np.abs(Ke)
        out = np.zeros((2 * len(nodes), X.shape[1]), dtype=np.complex128)
        for r, I in enumerate(nodes):
            cells, locs = np.nonzero(mesh.conn == I)
            for e, l in zip(cells, locs):
                J = mesh.conn[e]
                for al in range(2):
                    out[2 * r + al] += Ke[l] @ X[2 * J + al]
            for al in range(2):
                for be in range(2):
                    blk = (self.pv[I] if al == be else 0.0) + sum(self.pb[d][I] * PAULI[d][al, be]
                                                                for d in range(3))
                    out[2 * r + al] += (abs(blk) if magnitudes else blk) * X[2 * I + be]
        for pr in self.projectors:
            P, D = (np.abs(pr["P"]), np.abs(pr["Delta"])) if magnitudes else (pr["P"], pr["Delta"])
            C = D @ (P.T @ X[pr["rows"]])
            pos = {int(I): k for k, I in enumerate(pr["support"])}
            for r, I in enumerate(nodes):
                k = pos.get(int(I))
                if k is not None:
                    out[2 * r:2 * r + 2] += P[2 * k:2 * k + 2] @ C
        return out

    def dense(self) -> np.ndarray:
        """Dense H (tiny meshes only)."""
        H = self.Hloc.toarray()
        for pr in self.projectors:
            r = pr["rows"]
            H[np.ix_(r, r)] += pr["P"] @ pr["Delta"] @ pr["P"].T
        return H

    # -- derivatives -------------------------------------------------------
    def bilinear_grads(self, W: np.ndarray, U: np.ndarray, weight: float = 1.0):
        """Node-level derivatives of weight * Re tr(W^H H U).

        Returns (gV[M], gB[3, M], gh[natoms, 2]) where, for the quadrature
        point (e, l) mapped to node I, d/dV_{e,l} = w_l |J| gV[I] and
        d/dB_{d,e,l} = w_l |J| gB[d, I]; gh are derivatives in the couplings.
        """
        W2 = W.reshape(self.nnodes, 2, -1)
        U2 = U.reshape(self.nnodes, 2, -1)
        gV = weight * np.real(np.sum(np.conj(W2) * U2, axis=(1, 2)))
        gB = np.empty((3, self.nnodes))
        for d in range(3):
            SU = np.einsum("ab,Ibj->Iaj", PAULI[d], U2)
            gB[d] = weight * np.real(np.sum(np.conj(W2) * SU, axis=(1, 2)))
        gh = np.zeros((len(self.projectors), 2))
        for a, pr in enumerate(self.projectors):
            CW = pr["P"].T @ W[pr["rows"]]
            CU = pr["P"].T @ U[pr["rows"]]
            for j in range(2):
                gh[a, j] = weight * np.real(np.sum(np.conj(CW) * (channel_projector(j) @ CU)))
        return gV, gB, gh

    def node_to_quadrature(self, g_node: np.ndarray) -> np.ndarray:
        """Map node-level derivatives to per-quadrature-point ones: w_l |J| g[conn[e, l]]."""
        return self.mesh.quad_weights()[None, :] * g_node[self.mesh.conn]
