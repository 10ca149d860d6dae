"""Pins of the oracle's block FGMRES (no GPU): what block GMRES must do, checked
independently of its own recurrence."""
import numpy as np
import pytest

import workloads as W
from oracle import block_fgmres as BF
from oracle import elastic, fgmres, precond


def rand_system(n, seed, shift=4.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return A + shift * np.sqrt(n) * np.eye(n)


def test_cholqr2_orthonormal_factor_and_fallback():
    rng = np.random.default_rng(1)
    W = rng.standard_normal((200, 6)) + 1j * rng.standard_normal((200, 6))
    W[:, 5] = W[:, 0] * (1 + 1e-9) + 1e-13 * W[:, 1]          # nearly dependent column
    Q, R = BF.cholqr2(W)
    assert np.allclose(Q.conj().T @ Q, np.eye(6), atol=1e-12)
    assert np.allclose(Q @ R, W, atol=1e-10 * np.abs(W).max())
    assert np.allclose(np.tril(R, -1), 0.0)


def test_one_column_equals_fgmres():
    """s = 1: the block method is FGMRES (same Krylov space, same minimisation):
    the same iterate after k steps and the same count to a tolerance."""
    H = rand_system(60, 2, shift=1.5)
    b = np.random.default_rng(3).standard_normal(60) + 0j
    for k in (3, 9, 20):
        a = BF.block_fgmres(lambda V: H @ V, b, restart=10, rtol=1e-14, maxit=k)
        r = fgmres.fgmres(lambda v: H @ v, b, restart=10, rtol=1e-14, maxit=k)
        assert a.iters == r.iters == k
        assert np.linalg.norm(a.X[:, 0] - r.x) <= 1e-10 * np.linalg.norm(r.x)


def test_minimises_over_the_block_krylov_space():
    """After j unrestarted steps (identity preconditioner), column k's residual
    is the minimum of ||b_k - H x|| over x in the block Krylov space
    span{B, H B, ..., H^{j-1} B}, formed explicitly here and solved by least
    squares."""
    n, s = 40, 3
    H = rand_system(n, 4, shift=1.0)
    B = np.random.default_rng(5).standard_normal((n, s)) + 1j * np.random.default_rng(6).standard_normal((n, s))
    for j in (1, 2, 4, 6):
        res = BF.block_fgmres(lambda V: H @ V, B, restart=50, rtol=1e-15, maxit=j)
        K = np.column_stack([np.linalg.matrix_power(H, i) @ B for i in range(j)])
        K, _ = np.linalg.qr(K)
        HK = H @ K
        for c in range(s):
            y, *_ = np.linalg.lstsq(HK, B[:, c], rcond=None)
            best = np.linalg.norm(B[:, c] - HK @ y)
            got = np.linalg.norm(B[:, c] - H @ res.X[:, c])
            assert abs(got - best) <= 1e-9 * np.linalg.norm(B[:, c]), (j, c, got, best)


def test_decoupled_blocks_are_independent_gmres_runs():
    """H = diag(H1, H2) with B = [[b1, 0], [0, b2]]: the block Krylov space splits
    into the two single ones, so block GMRES gives the iterates of two separate
    GMRES runs."""
    H1, H2 = rand_system(30, 7, 1.2), rand_system(25, 8, 1.2)
    H = np.block([[H1, np.zeros((30, 25))], [np.zeros((25, 30)), H2]])
    rng = np.random.default_rng(9)
    b1 = rng.standard_normal(30) + 0j
    b2 = rng.standard_normal(25) + 0j
    B = np.zeros((55, 2), complex)
    B[:30, 0] = b1
    B[30:, 1] = b2
    for k in (2, 5, 8):
        a = BF.block_fgmres(lambda V: H @ V, B, restart=50, rtol=1e-15, maxit=k)
        r1 = fgmres.fgmres(lambda v: H1 @ v, b1, restart=50, rtol=1e-15, maxit=k)
        r2 = fgmres.fgmres(lambda v: H2 @ v, b2, restart=50, rtol=1e-15, maxit=k)
        assert np.linalg.norm(a.X[:30, 0] - r1.x) <= 1e-10 * np.linalg.norm(r1.x)
        assert np.linalg.norm(a.X[30:, 1] - r2.x) <= 1e-10 * np.linalg.norm(r2.x)
        assert np.abs(a.X[30:, 0]).max() <= 1e-12 and np.abs(a.X[:30, 1]).max() <= 1e-12


def test_finite_termination():
    """Unrestarted, the block Krylov space grows by s per step, so an N x N
    system is solved in at most ceil(N / s) steps."""
    n, s = 24, 4
    H = rand_system(n, 10, shift=0.5)
    B = np.random.default_rng(11).standard_normal((n, s)) + 0j
    res = BF.block_fgmres(lambda V: H @ V, B, restart=50, rtol=1e-10, maxit=50)
    assert res.converged and res.iters <= n // s


def test_block_with_the_multigrid_preconditioner_on_the_elastic_system():
    """Four point sources of a small layered medium, the block-acoustic multigrid
    preconditioner (a fixed cycle, hence a linear M): every column meets the
    tolerance by the assembled operator, and the block method needs no more
    iterations than the slowest of the four separate FGMRES solves (its space
    contains each of theirs)."""
    p = W.layered(64, 32, 4, seed=23, abc=6, nsrc=4, src_spacing=12)
    S = elastic.from_problem(p)
    pc = precond.multigrid(S, 3, precond.default_alpha(3))
    Bc = np.column_stack([W.padded_to_compact(W.point_source(p, q), p.n) for q in p.sources])
    Mb = lambda V: np.column_stack([pc.apply(V[:, c]) for c in range(V.shape[1])])
    res = BF.block_fgmres(lambda V: S.H @ V, Bc, Mb, restart=20, rtol=1e-6, maxit=400)
    assert res.converged
    rr = np.linalg.norm(Bc - S.H @ res.X, axis=0) / np.linalg.norm(Bc, axis=0)
    assert rr.max() <= 1e-6
    singles = [fgmres.fgmres(lambda v: S.H @ v, Bc[:, c], pc.apply, restart=20, rtol=1e-6, maxit=400).iters
               for c in range(4)]
    assert res.iters <= max(singles), (res.iters, singles)
