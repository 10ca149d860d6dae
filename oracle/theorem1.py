"""Spectral radius of the block-acoustic error iteration (Sec. 3, Theorem 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

With the distributed matrix K = D H (Eq. 3.3) and the block-triangular P
(Eq. 3.5), the error iteration of the preconditioned fixed-point method is
T = I - P^{-1} K.  Theorem 1 states that, with the exact blocks A and H_p in P,
spec(T) = spec(Z) u {0} for Z = Xi A^{-1} B^T H_p^{-1}, where Xi = B A - A_p B is
the commutator (Eq. 3.2), so rho(T) = rho(Z).  The paper estimates rho(Z) by
the power method on a matrix-free product with Z; ``rho_Z`` does that, with the
blocks shifted by alpha (Eq. 2.8) and solved by sparse LU.  ``power_T`` runs
the power method on T for any preconditioner given as a function, which is how
the GPU library measures the same quantity.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .elastic import ElasticSystem


def power(apply, x0, iters):
    """Power method: x_{k+1} = M x_k / ||M x_k|| from x0 / ||x0||; returns the
    history ||M x_k|| (k = 0 .. iters-1) and the estimate, the geometric mean
    of the last quarter of the history."""
    x = np.asarray(x0, dtype=np.complex128)
    x = x / np.linalg.norm(x)
    hist = []
    for _ in range(iters):
        y = apply(x)
        nrm = float(np.linalg.norm(y))
        hist.append(nrm)
        if nrm == 0.0:
            break
        x = y / nrm
    k = max(1, len(hist) // 4)
    return float(np.exp(np.mean(np.log(np.maximum(hist[-k:], 1e-300))))), np.asarray(hist)


def power_T(sys: ElasticSystem, apply_prec, x0, iters):
    """rho(T), T = I - P^{-1} D H, with apply_prec(r) = P^{-1} D r."""
    H = sys.H
    return power(lambda x: x - apply_prec(H @ x), x0, iters)


def rho_Z(sys: ElasticSystem, alpha, x0, iters, shift_sign=1.0):
    """rho(Z), Z = Xi A_s^{-1} B^T H_p,s^{-1} (Theorem 1), x0 on the pressure
    space; A_s and H_p,s are the blocks shifted by alpha (Eq. 2.8), Xi the
    commutator of the unshifted system."""
    d = sys.dim
    nu = sum(sys.sizes[:d])
    As = sp.block_diag([sys.A_shifted(k, alpha, shift_sign) for k in range(d)], format="csc")
    Hps = sp.csc_matrix(sys.Hp_shifted(alpha, shift_sign))
    Xi = sys.commutator()
    luA = spla.splu(As)
    luH = spla.splu(Hps)
    Bt = sys.Bt

    def Z(v):
        return Xi @ luA.solve(Bt @ luH.solve(v))

    assert len(x0) == sys.sizes[d] and As.shape[0] == nu
    return power(Z, x0, iters)
