"""Geometric multigrid for one acoustic block (Sec. 2.2, Algorithm 1, Sec. 4.4.1).

Paper passages followed:
  * Algorithm 1 (two-grid cycle), applied recursively with one recursive call
    (V-cycle) or two (W-cycle), Sec. 2.2.
  * Damped Jacobi relaxation with weights 0.8, 0.8, 0.3 on the first three
    levels (Sec. 4.4.1); the last weight is reused on deeper levels.
  * Restrictions, Eq. 4.1 / 4.2: Kronecker products of 1/4[1 2 1] along a
    nodal (face) direction and 1/8[1 3 * 3 1] along a cell-centred direction.
    "Mixed" restriction, Eq. 4.4: 1/2[1 * 1] along cell-centred directions.
  * Prolongation P proportional to R^T (Sec. 4.4.1) and Galerkin coarsening
    A_c = R A P (Eq. 4.3); the coarsest level is solved directly.

Readings:
  R7  P is bilinear interpolation (rows sum to one) and R = P^T / 2^d, which
      reproduces the printed stencils in the interior.  The paper's factor
      P = 2 R^T differs from the 2-D bilinear scale 4 R^T only by a constant,
      which cancels in P (R A P)^{-1} R and in Jacobi.  At the boundary, nodal
      directions use the zero normal displacement (the missing coarse face is
      zero) and cell-centred directions extrapolate the nearest coarse value
      (constant extrapolation).
  R9  default cycle V(1,2) in 2D (the paper uses W(1,2); a W flag exists).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .elastic import kron_axes
from .bf16 import round_matrix_bf16


# ----------------------------------------------------------------------------
# 1-D transfers
# ----------------------------------------------------------------------------
def prolong_nodal_1d(n):
    """(n-1, n/2-1): interior faces of a coarse line of n/2 cells -> interior
    faces of the fine line of n cells.  Coarse face K sits on fine face 2K;
    odd fine faces take the mean of their two coarse neighbours (a missing
    neighbour is the zero boundary face)."""
    nc = n // 2
    rows, cols, vals = [], [], []
    for K in range(1, nc):
        f = 2 * K
        rows.append(f - 1); cols.append(K - 1); vals.append(1.0)
        rows.append(f - 2); cols.append(K - 1); vals.append(0.5)
        rows.append(f);     cols.append(K - 1); vals.append(0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n - 1, nc - 1))


def prolong_cell_1d(n):
    """(n, n/2): cell-centred bilinear interpolation.  Fine cell 2J gets
    3/4 c_J + 1/4 c_{J-1}, fine cell 2J+1 gets 3/4 c_J + 1/4 c_{J+1}; a missing
    neighbour is replaced by c_J (constant extrapolation)."""
    nc = n // 2
    rows, cols, vals = [], [], []
    for J in range(nc):
        for f, Jn in ((2 * J, J - 1), (2 * J + 1, J + 1)):
            rows.append(f); cols.append(J); vals.append(0.75)
            rows.append(f); cols.append(Jn if 0 <= Jn < nc else J); vals.append(0.25)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, nc))


def restrict_cell_mixed_1d(n):
    """(n/2, n): the lower-order restriction 1/2[1 * 1] of Eq. 4.4."""
    nc = n // 2
    rows, cols, vals = [], [], []
    for J in range(nc):
        rows += [J, J]; cols += [2 * J, 2 * J + 1]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nc, n))


def block_kinds(d, block):
    """Per-axis location kind of an acoustic block: 'n' (nodal / face) or 'c'
    (cell).  block k < d is u_{k+1} (nodal along x_k), block d is p."""
    return ['n' if (a == block) else 'c' for a in range(d)]


def transfers(n, kinds, intergrid="bilinear"):
    """(P, R) between the fine grid of ``n`` cells and the grid of n/2 cells for
    a block whose per-axis kinds are ``kinds``."""
    d = len(n)
    Ps, Rs = [], []
    for a in range(d):
        if kinds[a] == 'n':
            p1 = prolong_nodal_1d(n[a])
            Ps.append(p1); Rs.append(sp.csr_matrix(p1.T) * 0.5)
        else:
            p1 = prolong_cell_1d(n[a])
            Ps.append(p1)
            if intergrid == "mixed":
                Rs.append(restrict_cell_mixed_1d(n[a]))
            else:
                Rs.append(sp.csr_matrix(p1.T) * 0.5)
    return kron_axes(Ps), kron_axes(Rs)


# ----------------------------------------------------------------------------
# hierarchy and cycle
# ----------------------------------------------------------------------------
DEFAULT_JACOBI = (0.8, 0.8, 0.3)


def jacobi_weight(level, weights=DEFAULT_JACOBI):
    return weights[min(level, len(weights) - 1)]


@dataclass
class Hierarchy:
    """Operators of one acoustic block on every level.  ``ops[l]`` is used in
    the relaxation and residual on level l, ``ops_exact[l]`` is the FP64
    Galerkin operator from which level l+1 is built and, on the coarsest level,
    the matrix that is solved directly."""
    ops: list
    ops_exact: list
    P: list
    R: list
    grids: list
    weights: tuple = DEFAULT_JACOBI
    nu_pre: int = 1
    nu_post: int = 2
    cycle: str = "V"
    coarse_lu: object = None
    diag: list = field(default_factory=list)

    @property
    def levels(self):
        return len(self.ops)


def build_hierarchy(A, n, kinds, levels, *, weights=DEFAULT_JACOBI, nu_pre=1, nu_post=2,
                    cycle="V", intergrid="bilinear", bf16=False):
    """Galerkin hierarchy A_{l+1} = R_l A_l P_l (Eq. 4.3) with ``levels`` levels
    (the fine level included).  With ``bf16`` the operators used for
    relaxation and residuals on levels 0..L-2 have every stored entry rounded
    to bfloat16 (real and imaginary parts separately), while the Galerkin
    products and the coarsest direct solve use the unrounded FP64 operators."""
    ops_exact, P, R, grids = [sp.csr_matrix(A)], [], [], [tuple(n)]
    cur = tuple(n)
    for _ in range(levels - 1):
        if any(v % 2 for v in cur) or min(cur) < 4:
            raise ValueError(f"cannot coarsen grid {cur}")
        Pl, Rl = transfers(cur, kinds, intergrid)
        P.append(Pl); R.append(Rl)
        ops_exact.append(sp.csr_matrix(Rl @ ops_exact[-1] @ Pl))
        cur = tuple(v // 2 for v in cur)
        grids.append(cur)
    ops = [round_matrix_bf16(o) if (bf16 and l < levels - 1) else o for l, o in enumerate(ops_exact)]
    hier = Hierarchy(ops, ops_exact, P, R, grids, tuple(weights), nu_pre, nu_post, cycle)
    hier.diag = [o.diagonal() for o in ops]
    hier.coarse_lu = spla.splu(sp.csc_matrix(ops_exact[-1]))
    return hier


def relax(A, diag, b, x, w):
    """One damped Jacobi sweep x <- x + w D^{-1} (b - A x)."""
    return x + w * (b - A @ x) / diag


def cycle(hier: Hierarchy, b, level=0, x=None):
    """Algorithm 1 applied recursively: pre-relax, restrict the residual, solve
    the coarse problem (recursively, once for V and twice for W), correct, and
    post-relax.  The coarsest level is solved directly."""
    if level == hier.levels - 1:
        return hier.coarse_lu.solve(b)
    A, dg = hier.ops[level], hier.diag[level]
    w = jacobi_weight(level, hier.weights)
    if x is None:
        x = np.zeros_like(b)
    for _ in range(hier.nu_pre):
        x = relax(A, dg, b, x, w)
    rc = hier.R[level] @ (b - A @ x)
    ec = cycle(hier, rc, level + 1)
    if hier.cycle == "W" and level + 1 < hier.levels - 1:
        ec = cycle(hier, rc, level + 1, ec)
    x = x + hier.P[level] @ ec
    for _ in range(hier.nu_post):
        x = relax(A, dg, b, x, w)
    return x
