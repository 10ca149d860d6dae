"""Block-acoustic preconditioner (Sec. 3, Eq. 3.1 - 3.5).

The distributor D = [[I, 0], [B, -A_p]] applied to H gives the distributed
system K = D H = [[A, B^T], [Xi, H_p]] (Eq. 3.3).  The preconditioner is the
block upper-triangular P = [[A, B^T], [0, H_p]] (Eq. 3.5), and one
preconditioning step maps a residual r = (r_u, r_p) to e = P^{-1} D r:

    t_p = B r_u - A_p r_p                 (right-hand side of Eq. 3.3, 2nd row)
    e_p = H_p^{-1} t_p                    (acoustic block, pressure velocity)
    e_u = A^{-1} (r_u - B^T e_p)          (d acoustic blocks, shear velocity)

The inverses are either exact (sparse LU, the setting of the scalability
table in Sec. 4.1) or approximate: one multigrid cycle per block on the
shifted operators of Eq. 2.8 (Sec. 4.4.1).

``precision='mixed'`` builds the same preconditioner from bfloat16-rounded
stored entries (A_p and every relaxation/residual operator above the coarsest
level), the rounding the mixed-precision GPU preconditioner applies to its
coefficient arrays; the arithmetic here stays FP64.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .bf16 import round_matrix_bf16
from .elastic import ElasticSystem
from . import multigrid as mg


ALPHA_BY_LEVELS = {1: 0.0, 2: 0.1, 3: 0.2, 4: 0.4}


ALPHA_DEEP = 1.0


def default_alpha(levels):
    """Shift by level count following the 2D linear-media table (Sec. 4.4.3):
    2 levels 0.1, 3 levels 0.2, 4 levels 0.4.  The paper's tables stop at 4
    levels and pick each shift by a search at resolution 0.1; deeper
    hierarchies use 1.0, the value such a search gives on the layered and
    random-field workloads with 5-7 levels."""
    return ALPHA_BY_LEVELS.get(levels, ALPHA_DEEP)


@dataclass
class BlockAcoustic:
    sys: ElasticSystem
    Ap: sp.csr_matrix
    B: sp.csr_matrix
    Bt: sp.csr_matrix
    solvers: list          # d+1 callables: block k -> approximate inverse of block k (k = d is H_p)
    sizes: list
    hier: list = None

    def apply(self, r):
        """e = P^{-1} D r (Eq. 3.3 - 3.5)."""
        d = self.sys.dim
        nu = sum(self.sizes[:d])
        r_u, r_p = r[:nu], r[nu:]
        t_p = self.B @ r_u - self.Ap @ r_p
        e_p = self.solvers[d](t_p)
        s_u = r_u - self.Bt @ e_p
        parts, off = [], 0
        for k in range(d):
            m = self.sizes[k]
            parts.append(self.solvers[k](s_u[off:off + m]))
            off += m
        parts.append(e_p)
        return np.concatenate(parts)


def _blocks(sys: ElasticSystem, alpha, shift_sign):
    d = sys.dim
    return [sys.A_shifted(k, alpha, shift_sign) for k in range(d)] + [sys.Hp_shifted(alpha, shift_sign)]


def exact(sys: ElasticSystem, alpha=0.0, shift_sign=1.0) -> BlockAcoustic:
    """Block-acoustic preconditioner with every block solved directly."""
    blocks = _blocks(sys, alpha, shift_sign)
    solvers = []
    for M in blocks:
        lu = spla.splu(sp.csc_matrix(M))
        solvers.append(lu.solve)
    return BlockAcoustic(sys, sys.Ap, sys.B, sys.Bt, solvers, sys.sizes)


def multigrid(sys: ElasticSystem, levels, alpha=None, *, weights=mg.DEFAULT_JACOBI, nu_pre=1, nu_post=2,
              cycle="V", intergrid="bilinear", precision="fp64", shift_sign=1.0, bf16_ap=None) -> BlockAcoustic:
    """Block-acoustic multigrid: one cycle of shifted-Laplacian multigrid per
    block (Sec. 4.4.1), with ``levels`` levels (fine level included).
    ``precision='mixed'`` rounds the level operators below the coarsest to
    bfloat16; ``bf16_ap`` says whether the distributor's A_p (Eq. 3.2) is
    rounded too (default: as the level operators; the 3-D GPU path keeps its
    distributor coefficients in FP64)."""
    if alpha is None:
        alpha = default_alpha(levels)
    d = sys.dim
    blocks = _blocks(sys, alpha, shift_sign)
    bf16 = precision == "mixed"
    hiers, solvers = [], []
    for k, M in enumerate(blocks):
        h = mg.build_hierarchy(M, sys.n, mg.block_kinds(d, k), levels, weights=weights, nu_pre=nu_pre,
                               nu_post=nu_post, cycle=cycle, intergrid=intergrid, bf16=bf16)
        hiers.append(h)
        solvers.append(lambda b, h=h: mg.cycle(h, b))
    if bf16_ap is None:
        bf16_ap = bf16
    Ap = round_matrix_bf16(sys.Ap) if bf16_ap else sys.Ap
    pc = BlockAcoustic(sys, Ap, sys.B, sys.Bt, solvers, sys.sizes, hiers)
    return pc


def dense_matrices(sys: ElasticSystem, alpha=0.0):
    """Dense P (Eq. 3.5), D (Eq. 3.1) and K = D H (Eq. 3.3) for tiny grids."""
    d = sys.dim
    blocks = _blocks(sys, alpha, 1.0)
    A = sp.block_diag(blocks[:d]).toarray()
    Hp = blocks[d].toarray()
    Bt = sys.Bt.toarray()
    B = sys.B.toarray()
    nu, npp = A.shape[0], Hp.shape[0]
    P = np.block([[A, Bt], [np.zeros((npp, nu)), Hp]])
    D = np.block([[np.eye(nu), np.zeros((nu, npp))], [B, -sys.Ap.toarray()]])
    K = D @ sys.H.toarray()
    return P, D, K
