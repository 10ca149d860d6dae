"""Adjoint gradient of a least-squares receiver misfit with respect to the
medium (lambda, mu, rho), for the mixed elastic Helmholtz operator H of
Eq. 2.6.  The paper solves the forward problem for full-waveform inversion
(Sec. 4) but does not write the gradient; this is the standard adjoint-state
derivation for the discrete system.

Misfit over sources s:  J = 1/2 sum_s || Q x_s - d_s ||^2,  H x_s = b_s, where
Q samples chosen entries (receivers) of the solution.  With
H^H y_s = Q^H (Q x_s - d_s):

    dJ/dm_k = - Re sum_s  y_s^H (dH/dm_k) x_s .

dH/dm_k is assembled from the same 1-D difference and averaging matrices as H
(Eq. 2.6): lambda enters only through -C = -diag(1/(lambda+mu)); mu enters
through A_e(mu) in the displacement blocks and through C; rho enters through
the face mass A_f(rho (1 - i gamma/omega)).  The oracle builds dH/dm_k for
every cell k (tiny grids) and uses sparse direct solves.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .elastic import (ElasticSystem, avg_cells_to_faces, d_cells_to_faces, d_faces_to_cells, eye, kron_axes)


def dH_dm(sys: ElasticSystem, param: str, k: int):
    """Sparse dH/dm_k for param in {'lambda', 'mu', 'rho'} (unshifted H)."""
    n, h, d = sys.n, sys.h, sys.dim
    N = sys.ncells
    e = np.zeros(N)
    e[k] = 1.0
    lm = sys.lam + sys.mu
    nu = sum(sys.sizes[:d])
    blocks_A = []
    if param in ("mu", "rho"):
        for c in range(d):
            if param == "mu":
                Dcc = kron_axes([d_faces_to_cells(n[a], h[a]) if a == c else eye(n[a]) for a in range(d)])
                Ac = Dcc.T @ sp.diags(e) @ Dcc
                for j in range(d):
                    if j == c:
                        continue
                    Dcj = kron_axes([eye(n[a] - 1) if a == c else (d_cells_to_faces(n[a], h[a]) if a == j else eye(n[a]))
                                     for a in range(d)])
                    Ae = kron_axes([avg_cells_to_faces(n[a]) if a in (c, j) else eye(n[a]) for a in range(d)])
                    Ac = Ac + Dcj.T @ sp.diags(Ae @ e) @ Dcj
            else:
                Af = kron_axes([avg_cells_to_faces(n[a]) if a == c else eye(n[a]) for a in range(d)])
                Ac = -sys.omega ** 2 * sp.diags(Af @ (e * (1.0 - 1j * sys.gamma / sys.omega)))
            blocks_A.append(sp.csr_matrix(Ac, dtype=np.complex128))
        dA = sp.block_diag(blocks_A, format="csr")
    else:
        dA = sp.csr_matrix((nu, nu), dtype=np.complex128)
    if param in ("lambda", "mu"):
        dC = sp.diags(e / lm ** 2)          # d(-C)/dm_k = + e_k e_k^T / (lambda+mu)^2
    else:
        dC = sp.csr_matrix((N, N))
    return sp.bmat([[dA, None], [None, dC]], format="csr")


def receiver_rows(sys: ElasticSystem, rec_cells):
    """Compact indices of the u_d unknowns at the given (i1, .., i_d) face
    indices (the receivers sample the last displacement component)."""
    d = sys.dim
    off = sum(sys.sizes[:d - 1])
    n = sys.n
    rows = []
    for c in rec_cells:
        # u_d lives on faces 1..n_d-1 along x_d, cells along the other axes
        idx = 0
        stride = 1
        for a in range(d):
            ia = c[a] - 1 if a == d - 1 else c[a]
            idx += ia * stride
            stride *= (n[a] - 1) if a == d - 1 else n[a]
        rows.append(off + idx)
    return np.asarray(rows)


def forward(sys: ElasticSystem, B):
    """Direct solves x_s = H^{-1} b_s (columns of B)."""
    lu = spla.splu(sp.csc_matrix(sys.H))
    return np.column_stack([lu.solve(B[:, s]) for s in range(B.shape[1])])


def misfit(sys: ElasticSystem, B, D, rows):
    X = forward(sys, B)
    R = X[rows, :] - D
    return 0.5 * float(np.sum(np.abs(R) ** 2)), X


def gradient(sys: ElasticSystem, B, D, rows, params=("lambda", "mu", "rho")):
    """(J, {param: dJ/dm}) by the adjoint state, dH/dm_k assembled per cell."""
    H = sp.csc_matrix(sys.H)
    lu = spla.splu(H)
    luH = spla.splu(sp.csc_matrix(H.conj().T))
    X = np.column_stack([lu.solve(B[:, s]) for s in range(B.shape[1])])
    R = X[rows, :] - D
    J = 0.5 * float(np.sum(np.abs(R) ** 2))
    Y = np.zeros_like(X)
    for s in range(B.shape[1]):
        rhs = np.zeros(H.shape[0], dtype=np.complex128)
        np.add.at(rhs, rows, R[:, s])       # Q^H r: a receiver listed twice contributes twice
        Y[:, s] = luH.solve(rhs)
    out = {}
    for prm in params:
        g = np.zeros(sys.ncells)
        for k in range(sys.ncells):
            dH = dH_dm(sys, prm, k)
            g[k] = -np.real(sum(np.vdot(Y[:, s], dH @ X[:, s]) for s in range(B.shape[1])))
        out[prm] = g
    return J, out, X, Y
