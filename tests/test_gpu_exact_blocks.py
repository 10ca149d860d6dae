"""The block-acoustic preconditioner with every acoustic block solved exactly
(Sec. 4.1, Table 2 uses this form to separate the preconditioner's quality
from the multigrid's).  Two GPU forms:

* the one-level hierarchy, whose "coarsest" level is the fine grid itself,
  inverted densely in FP64 at setup (grids up to 4096 cells per block);
* at any size, block_rtol > 0: every block solved to a relative residual
  block_rtol by an inner FP64 FGMRES preconditioned by its multigrid cycle,
  on the blocks shifted by block_alpha.

Pins: the GPU preconditioner equals the oracle's exact-block preconditioner
(sparse LU per block) to FP64 rounding amplified by the blocks' condition;
non-restarted FGMRES needs the oracle's iteration count (to within 1) on a
reduced linear medium (100x32, omega scaled to keep 10 points per shear
wavelength; the printed table starts at 200x64, whose dense inverses would
take the GPU about a minute to form)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import elastic, fgmres, precond

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_2411_15897_gb300 as bah  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def to_dev(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda")


def to_host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def linear_small():
    p = W.linear_medium(100, 32, 0.875 * math.pi, abc=10)
    return p, elastic.from_problem(p)


def test_exact_block_preconditioner_matches_oracle(linear_small):
    p, S = linear_small
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64, levels=1)
    assert s.levels == 1 and s.alpha == 0.0
    pc = precond.exact(S, 0.0)
    for seed in (51, 52):
        r = W.random_vector(p.n, seed)
        z = to_host(s.apply_preconditioner(to_dev(r)))
        assert rel(W.padded_to_compact(z, p.n), pc.apply(W.padded_to_compact(r, p.n))) <= 1e-8
    s.close()


@pytest.mark.parametrize("prec", [bah.BAH_FP64, bah.BAH_MIXED])
def test_exact_block_gmres_count(prec, linear_small):
    """Non-restarted (restart 50 > the count) FGMRES with exact block solves:
    the oracle's count, 19 here, within 1; every solve meets 1e-6 by the
    oracle's assembled operator."""
    p, S = linear_small
    b = W.point_source(p)
    bc = W.padded_to_compact(b, p.n)
    H = S.H
    ref = fgmres.fgmres(lambda v: H @ v, bc, precond.exact(S, 0.0).apply, restart=50, rtol=1e-6, maxit=200)
    assert ref.converged
    s = bah.Solver.from_problem(p, precision=prec, levels=1, restart=50, maxit=200)
    x, status, st = s.solve(to_dev(b), rtol=1e-6)
    assert status == bah.BAH_OK, st
    assert abs(st[0]["iters"] - ref.iters) <= 1, (st[0]["iters"], ref.iters)
    xc = W.padded_to_compact(to_host(x), p.n)
    assert np.linalg.norm(bc - H @ xc) / np.linalg.norm(bc) <= 1e-6
    s.close()


# ----------------------------------------------------------------------------
# spectral radius of T = I - P^{-1} D H (Sec. 3, Theorem 1) by the power method
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("levels,prec", [(1, bah.BAH_FP64), (3, bah.BAH_FP64), (3, bah.BAH_MIXED)])
def test_spectral_radius_matches_oracle_power_method(levels, prec, linear_small):
    """The same power method from the same start vector, on the GPU
    (bah_spectral_radius) and in the oracle (theorem1.power_T): with exact
    blocks (levels = 1) it estimates rho(T) = rho(Z) of Theorem 1; with
    multigrid blocks the fixed-point iteration's rate.  FP64 histories agree
    step by step; mixed precision to its rounding."""
    from oracle import theorem1
    p, S = linear_small
    x0 = W.random_vector(p.n, 53)
    s = bah.Solver.from_problem(p, precision=prec, levels=levels)
    rho, hist = bah.bah_spectral_radius(s.ctx, to_dev(x0), 60)
    pc = (precond.exact(S, 0.0) if levels == 1
          else precond.multigrid(S, levels, precond.default_alpha(levels),
                                 precision="fp64" if prec == bah.BAH_FP64 else "mixed"))
    ref, ref_hist = theorem1.power_T(S, pc.apply, W.padded_to_compact(x0, p.n), 60)
    tol = 1e-8 if prec == bah.BAH_FP64 else 1e-3
    np.testing.assert_allclose(hist, ref_hist, rtol=tol)
    assert abs(rho - ref) <= tol * ref
    s.close()


# ----------------------------------------------------------------------------
# exact blocks at any size: inner FGMRES block solves (block_rtol > 0)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [bah.BAH_FP64, bah.BAH_MIXED])
@pytest.mark.parametrize("balpha", [0.0, 0.3])
def test_inner_block_solves_equal_the_oracle_exact_blocks(prec, balpha, linear_small):
    """With block_rtol = 1e-12 the preconditioner is the oracle's exact-block
    preconditioner (sparse LU of each block shifted by block_alpha) to the
    inner tolerance amplified by the coupling B, B^T (FP64 mode), or to one
    FP32 rounding of the result (mixed mode, where the flexible basis is
    FP32); the multigrid hierarchy keeps its own shift."""
    p, S = linear_small
    s = bah.Solver.from_problem(p, precision=prec, block_rtol=1e-12, block_alpha=balpha)
    assert s.levels > 1
    pc = precond.exact(S, balpha)
    for seed in (61, 62):
        r = W.random_vector(p.n, seed)
        z = to_host(s.apply_preconditioner(to_dev(r)))
        err = rel(W.padded_to_compact(z, p.n), pc.apply(W.padded_to_compact(r, p.n)))
        assert err <= (1e-9 if prec == bah.BAH_FP64 else 1e-6), err
    info = bah.bah_get_info(s.ctx)
    assert info["block_iters"] > 0 and info["block_failures"] == 0
    s.close()


@pytest.mark.parametrize("grid,omega_pi", [((200, 64), 1.75), ((400, 128), 3.5)])
@pytest.mark.parametrize("lam", [1, 10, 100, 1000])
def test_table2_counts_with_exact_blocks(grid, omega_pi, lam):
    """Table 2's experiment on its two smaller grids: the linear medium with
    lambda scaled by 1, 10, 100, 1000, non-restarted FGMRES with every block
    solved exactly.  The GPU (inner block solves to 1e-9) needs the oracle's
    count (sparse LU per block) within 1, and every solve meets 1e-6 by the
    oracle's assembled operator."""
    p = W.linear_medium(grid[0], grid[1], omega_pi * math.pi, lam_factor=float(lam))
    S = elastic.from_problem(p)
    b = W.point_source(p)
    bc = W.padded_to_compact(b, p.n)
    H = S.H
    ref = fgmres.fgmres(lambda v: H @ v, bc, precond.exact(S, 0.0).apply, restart=64, rtol=1e-6, maxit=64)
    assert ref.converged
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64, restart=64, maxit=64, block_rtol=1e-9)
    x, status, st = s.solve(to_dev(b), rtol=1e-6)
    assert status == bah.BAH_OK, st
    print(f"Table 2 {grid[0]}x{grid[1]} lambda x{lam}: GPU {st[0]['iters']}, oracle {ref.iters}")
    assert abs(st[0]["iters"] - ref.iters) <= 1, (st[0]["iters"], ref.iters)
    xc = W.padded_to_compact(to_host(x), p.n)
    assert np.linalg.norm(bc - H @ xc) / np.linalg.norm(bc) <= 1e-6
    assert bah.bah_get_info(s.ctx)["block_failures"] == 0
    s.close()


def test_table2_scalability_on_the_large_grids():
    """The scalability claim of Table 2 on its two larger grids (800x256 and
    1600x512, omega doubled with each refinement), where only the GPU runs:
    with exact blocks the non-restarted count does not grow with the grid --
    it stays at or below the 200x64 count -- for lambda x 1 and x 1000, as in
    the printed table (14 -> 14; 13 -> 12).  True residuals by the library's
    FP64 residual."""
    counts = {}
    for (n1, n2, om) in ((200, 64, 1.75), (800, 256, 7.0), (1600, 512, 14.0)):
        for lam in (1, 1000):
            p = W.linear_medium(n1, n2, om * math.pi, lam_factor=float(lam))
            s = bah.Solver.from_problem(p, precision=bah.BAH_FP64, restart=64, maxit=64, block_rtol=1e-9)
            x, status, st = s.solve(to_dev(W.point_source(p)), rtol=1e-6)
            assert status == bah.BAH_OK, st
            assert st[0]["relres_true"] <= 1e-6
            assert bah.bah_get_info(s.ctx)["block_failures"] == 0
            counts[(n1, lam)] = st[0]["iters"]
            s.close()
    print("Table 2 on the GPU (non-restarted FGMRES, exact blocks):", counts)
    for lam in (1, 1000):
        for n1 in (800, 1600):
            assert counts[(n1, lam)] <= counts[(200, lam)], counts


@pytest.mark.parametrize("grid,omega_pi", [((200, 64), 1.75), ((400, 128), 3.5)])
@pytest.mark.parametrize("alpha", [0.0, 0.25, 0.5, 1.0])
def test_rho_z_against_shift_on_the_linear_medium(alpha, grid, omega_pi):
    """rho(Z) against the shift (Sec. 3, Theorem 1; the paper's rho(Z)
    experiment on the 400x128 linear medium, and on 200x64): the power method
    on a matrix-free product with Z = Xi A_s^{-1} B^T H_p,s^{-1}, the shifted
    blocks solved exactly (inner solves to 1e-12).  The GPU history equals the
    oracle's (sparse LU) step by step.  At alpha = 0 Theorem 1 gives
    rho(T) = rho(Z) for T = I - P^{-1} D H, which bah_spectral_radius checks."""
    from oracle import theorem1
    p = W.linear_medium(grid[0], grid[1], omega_pi * math.pi)
    S = elastic.from_problem(p)
    x0 = W.random_vector(p.n, 57)
    xp = W.padded_to_compact(x0, p.n)[-S.sizes[-1]:]
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64, block_rtol=1e-12, block_alpha=alpha)
    rho, hist = bah.bah_spectral_radius_z(s.ctx, to_dev(x0[-1]), 40)
    ref, ref_hist = theorem1.rho_Z(S, alpha, xp, 40)
    print(f"rho(Z) {grid[0]}x{grid[1]} alpha {alpha}: GPU {rho:.4f}, oracle {ref:.4f}")
    np.testing.assert_allclose(hist, ref_hist, rtol=1e-6)
    assert abs(rho - ref) <= 1e-6 * ref
    if alpha == 0.0:
        # Theorem 1: spec(T) = spec(Z) u {0}, so the power method on T tends to the
        # same radius (it converges more slowly on T: 80 steps, 5%)
        rt, _ = bah.bah_spectral_radius(s.ctx, to_dev(x0), 80)
        assert abs(rt - rho) <= 0.05 * rho, (rt, rho)
    s.close()
