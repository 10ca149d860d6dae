"""Flexible GMRES with right preconditioning (the outer Krylov solver the
paper uses, Sec. 2.2 and Sec. 4: FGMRES of Saad 1993; GMRES(5) and
non-restarted GMRES in the experiments).

Textbook form, written plainly:
  x_0 = 0 (or a given start),  r_0 = b - H x_0,  beta = ||r_0||,  v_1 = r_0/beta
  for j = 1..m:
      z_j = M_j(v_j)                   (preconditioner, may change every step)
      w   = H z_j
      h_{i,j} = v_i^H w,  w -= h_{i,j} v_i   for i = 1..j   (modified Gram-Schmidt)
      h_{j+1,j} = ||w||,  v_{j+1} = w / h_{j+1,j}
      y_j = argmin || beta e_1 - Hbar_j y ||   (numpy least squares)
      stop when that minimum <= rtol ||b||
  x = x_0 + Z_j y_j;  restart from x if the true residual is still above rtol ||b||.

Stopping reading (R12): 2-norm of the unpreconditioned residual relative to
||b||, x_0 = 0, confirmed by the true residual b - H x in FP64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Result:
    x: np.ndarray
    iters: int
    restarts: int
    relres_true: float
    relres_est: float
    converged: bool
    history: list = field(default_factory=list)     # estimated relative residual after each iteration


def fgmres(apply_H, b, precond=None, *, restart=20, rtol=1e-6, maxit=1000, x0=None, callback=None) -> Result:
    """Solve H x = b.  ``apply_H`` and ``precond`` are callables on 1-D complex
    vectors; ``precond=None`` is the identity (plain GMRES)."""
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return Result(np.zeros_like(b), 0, 0, 0.0, 0.0, True)
    M = precond if precond is not None else (lambda v: v.copy())
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - apply_H(x)
    beta = np.linalg.norm(r)
    total, restarts, hist = 0, 0, []
    est = beta / nb
    while True:
        if beta <= rtol * nb or total >= maxit:
            break
        m = min(restart, maxit - total)
        V = [r / beta]
        Z = []
        Hbar = np.zeros((m + 1, m), dtype=np.complex128)
        y = None
        for j in range(m):
            z = M(V[j])
            Z.append(z)
            w = apply_H(z)
            for i in range(j + 1):
                Hbar[i, j] = np.vdot(V[i], w)
                w = w - Hbar[i, j] * V[i]
            Hbar[j + 1, j] = np.linalg.norm(w)
            total += 1
            rhs = np.zeros(j + 2, dtype=np.complex128)
            rhs[0] = beta
            y, *_ = np.linalg.lstsq(Hbar[:j + 2, :j + 1], rhs, rcond=None)
            res = np.linalg.norm(rhs - Hbar[:j + 2, :j + 1] @ y)
            est = res / nb
            hist.append(est)
            if callback is not None:
                callback(total, est)
            breakdown = Hbar[j + 1, j] <= 1e-14 * np.linalg.norm(Hbar[:j + 2, j])
            if res <= rtol * nb or breakdown:
                break
            V.append(w / Hbar[j + 1, j])
        x = x + np.column_stack(Z) @ y
        r = b - apply_H(x)
        beta = np.linalg.norm(r)
        restarts += 1
    relres = beta / nb
    return Result(x, total, restarts, relres, est, relres <= rtol, hist)
