"""Discrete mixed elastic Helmholtz operator and the acoustic blocks of the
block-acoustic preconditioner, assembled as sparse FP64 matrices.

Paper passages followed:
  * Eq. 2.5 (mixed continuous system) and Eq. 2.6 (its MAC discretisation):
        H = [[A, B^T], [B, -C]],
        A = grad_h^T A_e(mu) grad_h - omega^2 M,   M = A_f(rho (1 - i gamma/omega)),
        B^T = grad_h,  C = diag(1/(lambda+mu)).
    u_k lives on the x_k-faces, p and the medium at cell centres (Fig. 1).
  * Eq. 3.2:  A_p = B B^T diag(mu) - omega^2 M_p,  M_p = diag(rho (1 - i gamma/omega)).
  * Eq. 3.4:  H_p = B B^T + A_p C.
  * Eq. 2.8 (complex shift, CSLP):  H_s = H - i alpha omega^2 M_s.

Readings where the paper is silent or ambiguous:
  R1  outer boundary: the displacement normal to the boundary is zero (those
      faces carry no unknown), and derivative terms that would sit on the
      boundary for tangential derivatives are dropped.  Hence B^T = grad_h maps
      cells to interior faces, B B^T is the cell Laplacian with zero-flux
      boundaries, and H is complex symmetric.
  R2  A_e(mu): arithmetic mean of the 2^2 cells around each edge (node in 2D);
      the own-direction derivative lands on the cell centre and uses that
      cell's mu.  A_f: arithmetic mean of the two cells sharing a face.
  R3  shift sign: Eq. 2.8 is written for the acoustic operator with the
      positive Laplacian; in the mixed system (negative Laplacian) the same
      damping is  + i alpha omega^2 M_s, i.e. gamma -> gamma + alpha*omega in each
      block's own mass term (the shift acts as added attenuation, Sec. 3.1).
      M_s = A_f(rho) for the displacement blocks and diag(rho/(lambda+mu)) for
      H_p.  ``shift_sign=-1`` gives the opposite reading for comparison.

Unknown ordering (compact): [u_1 | ... | u_d | p]; every component is x_1
fastest over its own unknowns (u_k: n_k-1 interior faces along x_k).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------------------
# 1-D building blocks on a line of n cells with spacing h
# ----------------------------------------------------------------------------
def d_faces_to_cells(n, h):
    """(n, n-1): derivative of a face field at the cell centres, the two
    boundary faces being zero (R1):  (D u)_i = (u_{i+1} - u_i) / h."""
    rows, cols, vals = [], [], []
    for i in range(n):
        if i >= 1:                      # lower face i  (column i-1)
            rows.append(i); cols.append(i - 1); vals.append(-1.0 / h)
        if i + 1 <= n - 1:              # upper face i+1 (column i)
            rows.append(i); cols.append(i); vals.append(1.0 / h)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n - 1))


def d_cells_to_faces(n, h):
    """(n-1, n): derivative of a cell field at the interior faces:
    (G p)_f = (p_f - p_{f-1}) / h, f = 1..n-1."""
    rows, cols, vals = [], [], []
    for f in range(1, n):
        rows += [f - 1, f - 1]; cols += [f - 1, f]; vals += [-1.0 / h, 1.0 / h]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n - 1, n))


def avg_cells_to_faces(n):
    """(n-1, n): arithmetic mean of the two cells sharing each interior face."""
    rows, cols, vals = [], [], []
    for f in range(1, n):
        rows += [f - 1, f - 1]; cols += [f - 1, f]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n - 1, n))


def kron_axes(mats):
    """Kronecker product of per-axis matrices ``mats[0]`` (x_1, fastest) ..
    ``mats[d-1]`` (x_d, slowest)."""
    out = sp.csr_matrix(mats[0])
    for m in mats[1:]:
        out = sp.kron(m, out, format="csr")
    return out


def eye(n):
    return sp.identity(n, format="csr")


# ----------------------------------------------------------------------------
# assembled system
# ----------------------------------------------------------------------------
@dataclass
class ElasticSystem:
    n: tuple
    h: tuple
    omega: float
    lam: np.ndarray      # flat, cells, x_1 fastest
    mu: np.ndarray
    rho: np.ndarray
    gamma: np.ndarray
    G: list              # G[k] = (B^T)_k : cells -> u_k faces
    A: list              # A[k] : displacement block k (Eq. 2.6)
    Afk: list            # face-averaging operators cells -> u_k faces
    C: sp.csr_matrix     # diag(1/(lambda+mu))
    sizes: list          # unknowns per component

    @property
    def dim(self):
        return len(self.n)

    @property
    def ncells(self):
        return int(np.prod(self.n))

    @property
    def rho_t(self):
        """rho (1 - i gamma/omega) at cells (Eq. 2.6)."""
        return self.rho * (1.0 - 1j * self.gamma / self.omega)

    # -- Eq. 2.6 ---------------------------------------------------------
    @property
    def Bt(self):
        return sp.vstack(self.G, format="csr")

    @property
    def B(self):
        return sp.csr_matrix(self.Bt.T)

    @property
    def Ablk(self):
        return sp.block_diag(self.A, format="csr")

    @property
    def H(self):
        """The mixed elastic Helmholtz matrix [[A, B^T], [B, -C]] (Eq. 2.6)."""
        return sp.bmat([[self.Ablk, self.Bt], [self.B, -self.C]], format="csr")

    # -- Eq. 3.2, 3.4 ----------------------------------------------------
    @property
    def BBt(self):
        return sp.csr_matrix(self.B @ self.Bt)

    @property
    def Ap(self):
        """A_p = B B^T diag(mu) - omega^2 diag(rho(1 - i gamma/omega)) (Eq. 3.2)."""
        return sp.csr_matrix(self.BBt @ sp.diags(self.mu) - self.omega ** 2 * sp.diags(self.rho_t))

    @property
    def Hp(self):
        """H_p = B B^T + A_p C (Eq. 3.4)."""
        return sp.csr_matrix(self.BBt + self.Ap @ self.C)

    # -- Eq. 2.8 shifted blocks (reading R3) -------------------------------
    def A_shifted(self, k, alpha, shift_sign=1.0):
        ms = self.Afk[k] @ self.rho
        return sp.csr_matrix(self.A[k] + shift_sign * 1j * alpha * self.omega ** 2 * sp.diags(ms))

    def Hp_shifted(self, alpha, shift_sign=1.0):
        ms = self.rho / (self.lam + self.mu)
        return sp.csr_matrix(self.Hp + shift_sign * 1j * alpha * self.omega ** 2 * sp.diags(ms))

    def commutator(self):
        """Xi = B A - A_p B (Eq. 2.10 / 3.3), mapping u -> cells."""
        return sp.csr_matrix(self.B @ self.Ablk - self.Ap @ self.B)


def assemble(n, h, lam, mu, rho, gamma, omega) -> ElasticSystem:
    """Assemble the mixed MAC system of Eq. 2.6 for a d-dimensional grid of
    ``n`` cells (x_1 first) with spacings ``h`` and cell-centred medium arrays
    in numpy order (shape (n_d, .., n_1))."""
    n = tuple(int(v) for v in n)
    h = tuple(float(v) for v in h)
    d = len(n)
    lam = np.asarray(lam, dtype=np.float64).ravel()
    mu = np.asarray(mu, dtype=np.float64).ravel()
    rho = np.asarray(rho, dtype=np.float64).ravel()
    gamma = np.asarray(gamma, dtype=np.float64).ravel()
    rho_t = rho * (1.0 - 1j * gamma / omega)

    G, A, Afk, sizes = [], [], [], []
    for k in range(d):
        # gradient of p onto the interior x_k-faces
        G.append(kron_axes([d_cells_to_faces(n[a], h[a]) if a == k else eye(n[a]) for a in range(d)]))
        # own-direction derivative of u_k, evaluated at cell centres with mu there
        Dkk = kron_axes([d_faces_to_cells(n[a], h[a]) if a == k else eye(n[a]) for a in range(d)])
        Ak = Dkk.T @ sp.diags(mu) @ Dkk
        # cross derivatives of u_k along x_j (j != k) at the interior (k,j)-edges
        for j in range(d):
            if j == k:
                continue
            Dkj = kron_axes([eye(n[a] - 1) if a == k else (d_cells_to_faces(n[a], h[a]) if a == j else eye(n[a]))
                             for a in range(d)])
            Ae = kron_axes([avg_cells_to_faces(n[a]) if a in (k, j) else eye(n[a]) for a in range(d)])
            mu_e = Ae @ mu
            Ak = Ak + Dkj.T @ sp.diags(mu_e) @ Dkj
        Af = kron_axes([avg_cells_to_faces(n[a]) if a == k else eye(n[a]) for a in range(d)])
        Ak = Ak - omega ** 2 * sp.diags(Af @ rho_t)
        A.append(sp.csr_matrix(Ak))
        Afk.append(sp.csr_matrix(Af))
        sizes.append(Af.shape[0])
    sizes.append(int(np.prod(n)))
    C = sp.diags(1.0 / (lam + mu)).tocsr()
    return ElasticSystem(n, h, float(omega), lam, mu, rho, gamma, G, A, Afk, C, sizes)


def from_problem(prob) -> ElasticSystem:
    """Assemble from a ``workloads.Problem``."""
    return assemble(prob.n, prob.h, prob.lam, prob.mu, prob.rho, prob.gamma, prob.omega)
