"""Block flexible GMRES for s right-hand sides at once (the batched form of
the outer solve; the paper's outer solver is FGMRES, Sec. 2.2 and Sec. 4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

One Krylov space is built for the whole block B = [b_1 .. b_s] (N x s):

  X_0 = 0,  R_0 = B - H X_0,  R_0 = V_0 S_0                 (QR of the block)
  for j = 0 .. m-1:
      Z_j = M(V_j)                  (the preconditioner on each column; may change per step)
      W   = H Z_j
      two passes of block classical Gram-Schmidt (CGS2):
          C = [V_0 .. V_j]^H W,   W -= [V_0 .. V_j] C,   Hbar[0..j, j] += C
      W = V_{j+1} R                 (QR of the new block by CholQR2)
      Hbar[j+1, j] = R
      Y = argmin || E_1 S_0 - Hbar_j Y ||_F   (numpy least squares, column by column)
      stop when every column's minimum <= rtol ||b_k||
  X = X_0 + [Z_0 .. Z_j] Y;  restart from X while a true residual is above rtol ||b_k||.

Each block is an N x s matrix and Hbar is block upper Hessenberg with s x s
blocks.  CholQR (Cholesky QR): G = W^H W, G = L L^H, Q = W L^{-H}, R = L^H;
CholQR2 applies it twice (Q, R1 = CholQR(W); Q', R2 = CholQR(Q); R = R2 R1),
which restores orthogonality to working precision when W is not too
ill-conditioned.  A block whose Gram matrix is singular (some columns already
converged, or a column dependence) is factorised by a Householder QR instead,
whose Q stays orthonormal; each column still minimises its residual over the
whole block Krylov space built so far.

Stopping reading (R12, per right-hand side): ||b_k - H x_k|| <= rtol ||b_k||,
confirmed by the true residual in FP64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class BlockResult:
    X: np.ndarray                    # N x s solutions
    iters: int                       # block iterations (preconditioner applications per column)
    restarts: int
    relres_true: np.ndarray          # per column
    relres_est: np.ndarray
    converged: bool
    history: list = field(default_factory=list)   # per block iteration: estimated relative residuals (s,)


def cholqr(W):
    """One Cholesky QR of the N x s block W: (Q, R) with W = Q R, R upper
    triangular.  Returns None when the Gram matrix is not numerically
    positive definite."""
    G = W.conj().T @ W
    G = 0.5 * (G + G.conj().T)
    try:
        L = np.linalg.cholesky(G)
    except np.linalg.LinAlgError:
        return None
    R = L.conj().T
    Q = np.linalg.solve(L, W.conj().T).conj().T          # W R^{-1}
    return Q, R


def cholqr2(W):
    """CholQR applied twice, (Q, R) with W = Q R; falls back to a Householder
    QR of the block (numpy), whose Q stays orthonormal, when the block is
    numerically rank deficient."""
    f1 = cholqr(W)
    if f1 is not None:
        Q1, R1 = f1
        f2 = cholqr(Q1)
        if f2 is not None:
            Q, R2 = f2
            return Q, R2 @ R1
    Q, R = np.linalg.qr(W)
    return Q, R


def block_fgmres(apply_H, B, precond=None, *, restart=20, rtol=1e-6, maxit=1000, X0=None) -> BlockResult:
    """Solve H X = B for the N x s block B; ``apply_H`` and ``precond`` act on
    N x s blocks (column by column); ``precond=None`` is the identity."""
    B = np.asarray(B, dtype=np.complex128)
    if B.ndim == 1:
        B = B[:, None]
    N, s = B.shape
    nb = np.linalg.norm(B, axis=0)
    nb_safe = np.where(nb > 0.0, nb, 1.0)
    M = precond if precond is not None else (lambda V: V.copy())
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.complex128)
    R0 = B - apply_H(X)
    beta = np.linalg.norm(R0, axis=0)
    total, restarts, hist = 0, 0, []
    est = beta / nb_safe
    while np.any(beta > rtol * nb) and total < maxit:
        m = min(restart, maxit - total)
        V0, S0 = cholqr2(R0)
        V = [V0]
        Z = []
        Hbar = np.zeros(((m + 1) * s, m * s), dtype=np.complex128)
        E1S0 = np.zeros(((m + 1) * s, s), dtype=np.complex128)
        E1S0[:s, :] = S0
        Y = None
        for j in range(m):
            Zj = M(V[j])
            Z.append(Zj)
            W = apply_H(Zj)
            Vcat = np.column_stack(V)                  # N x (j+1) s
            for _ in range(2):                         # CGS2
                C = Vcat.conj().T @ W
                W = W - Vcat @ C
                Hbar[:(j + 1) * s, j * s:(j + 1) * s] += C
            Vn, Rn = cholqr2(W)
            Hbar[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = Rn
            total += 1
            Hj = Hbar[:(j + 2) * s, :(j + 1) * s]
            rhs = E1S0[:(j + 2) * s, :]
            Y, *_ = np.linalg.lstsq(Hj, rhs, rcond=None)
            res = np.linalg.norm(rhs - Hj @ Y, axis=0)
            est = res / nb_safe
            hist.append(est.copy())
            if np.all(res <= rtol * nb) or total >= maxit:
                break
            V.append(Vn)
        X = X + np.column_stack(Z) @ Y
        R0 = B - apply_H(X)
        beta = np.linalg.norm(R0, axis=0)
        restarts += 1
    relres = beta / nb_safe
    return BlockResult(X, total, restarts, relres, est, bool(np.all(beta <= rtol * nb)), hist)
