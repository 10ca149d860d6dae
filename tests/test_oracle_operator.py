"""Pins of the oracle's discrete operators against what the paper and the
mathematics fix (no GPU).  Each test names the passage it checks."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import elastic

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def const_system(n, h, lam=3.0, mu=1.5, rho=1.2, gamma=0.7, omega=5.0):
    shape = tuple(reversed(n))
    f = lambda v: np.full(shape, float(v))
    return elastic.assemble(n, h, f(lam), f(mu), f(rho), f(gamma), omega)


def cos_mode(n, k):
    """Neumann (cell-centred) eigenvector of B B^T: prod_a cos(pi k_a (i_a+1/2)/n_a)."""
    grids = np.meshgrid(*[np.cos(math.pi * k[a] * (np.arange(n[a]) + 0.5) / n[a]) for a in reversed(range(len(n)))],
                        indexing="ij")
    return np.prod(grids, axis=0).ravel()


def lap_eig(n, h, k):
    return sum(4.0 / h[a] ** 2 * math.sin(math.pi * k[a] / (2 * n[a])) ** 2 for a in range(len(n)))


@pytest.mark.parametrize("n", [(7, 5), (4, 5, 6)])
def test_complex_symmetric(n):
    """Eq. 2.6 with B^T = grad_h and a symmetric A: H^T = H exactly (reading R1)."""
    p = W.random_medium(n, 3)
    S = elastic.from_problem(p)
    H = S.H
    assert abs(H - H.T).max() == 0.0
    assert H.shape[0] == sum(W.compact_sizes(n))


def test_block_eigen_closed_form_2d():
    """Constant medium: A_1 acts on sin(pi k1 i/n1) cos(pi k2 (j+1/2)/n2) with
    eigenvalue mu*lap - omega^2 rho(1 - i gamma/omega) (Eq. 2.6: Dirichlet
    normal displacement, zero-flux tangential derivatives, reading R1)."""
    n, h = (9, 7), (0.3, 0.2)
    lam, mu, rho, gam, om = 3.0, 1.5, 1.2, 0.7, 5.0
    S = const_system(n, h, lam, mu, rho, gam, om)
    rt = rho * (1 - 1j * gam / om)
    for k1, k2 in [(1, 0), (3, 2), (8, 6)]:
        # u1: faces i = 1..n1-1 along x (Dirichlet), cells j along z (Neumann)
        v = np.outer(np.cos(math.pi * k2 * (np.arange(n[1]) + 0.5) / n[1]),
                     np.sin(math.pi * k1 * np.arange(1, n[0]) / n[0])).ravel()
        ev = mu * (4 / h[0] ** 2 * math.sin(math.pi * k1 / (2 * n[0])) ** 2
                   + 4 / h[1] ** 2 * math.sin(math.pi * k2 / (2 * n[1])) ** 2) - om ** 2 * rt
        np.testing.assert_allclose(S.A[0] @ v, ev * v, rtol=0, atol=1e-11 * abs(ev) * np.abs(v).max())
    for kx, kz in [(0, 1), (4, 3), (8, 6)]:
        # u2: cells along x (Neumann), faces along z (Dirichlet)
        v2 = np.outer(np.sin(math.pi * kz * np.arange(1, n[1]) / n[1]),
                      np.cos(math.pi * kx * (np.arange(n[0]) + 0.5) / n[0])).ravel()
        ev2 = mu * (4 / h[0] ** 2 * math.sin(math.pi * kx / (2 * n[0])) ** 2
                    + 4 / h[1] ** 2 * math.sin(math.pi * kz / (2 * n[1])) ** 2) - om ** 2 * rt
        np.testing.assert_allclose(S.A[1] @ v2, ev2 * v2, rtol=0, atol=1e-11 * abs(ev2) * np.abs(v2).max())


@pytest.mark.parametrize("n,h,modes", [((8, 6), (0.25, 0.3), [(0, 0), (2, 1), (7, 5)]),
                                        ((6, 5, 4), (0.25, 0.3, 0.2), [(0, 0, 0), (2, 1, 3), (5, 4, 1)])])
def test_Hp_closed_form_pressure_velocity(n, h, modes):
    """Eq. 3.2 / 3.4 with a constant medium: (lambda+mu) H_p acts on the Neumann
    modes as (lambda+2mu) lap - omega^2 rho~, an acoustic operator with the
    pressure velocity Vp (Sec. 3), in 2-D and 3-D."""
    lam, mu, rho, gam, om = 3.0, 1.5, 1.2, 0.7, 5.0
    S = const_system(n, h, lam, mu, rho, gam, om)
    rt = rho * (1 - 1j * gam / om)
    for k in modes:
        v = cos_mode(n, k)
        ev = ((lam + 2 * mu) * lap_eig(n, h, k) - om ** 2 * rt) / (lam + mu)
        np.testing.assert_allclose(S.Hp @ v, ev * v, rtol=0, atol=1e-11 * (abs(ev) + 100))
        evp = mu * lap_eig(n, h, k) - om ** 2 * rt
        np.testing.assert_allclose(S.Ap @ v, evp * v, rtol=0, atol=1e-11 * (abs(evp) + 100))


@pytest.mark.parametrize("n", [(9, 8), (6, 5, 4)])
def test_Hp_identity_variable_medium(n):
    """H_p = B B^T + A_p C equals B B^T diag((lambda+2mu)/(lambda+mu)) -
    omega^2 diag(rho~/(lambda+mu)) (algebra of Eq. 3.2, 3.4), in 2-D and 3-D."""
    p = W.random_medium(n, 5)
    S = elastic.from_problem(p)
    rhs = S.BBt @ sp.diags((S.lam + 2 * S.mu) / (S.lam + S.mu)) - S.omega ** 2 * sp.diags(S.rho_t / (S.lam + S.mu))
    assert abs(S.Hp - rhs).max() < 1e-9 * abs(rhs).max()


@pytest.mark.parametrize("n,h,modes", [((8, 7), (0.2, 0.25), [(1, 0), (3, 4), (6, 6)]),
                                        ((6, 5, 4), (0.2, 0.25, 0.3), [(1, 0, 0), (3, 4, 2), (5, 1, 3)])])
def test_mu0_reduction_to_acoustic(n, h, modes):
    """Eq. 2.4: with mu = 0 the elastic system reduces to an acoustic Helmholtz
    equation with velocity sqrt(lambda/rho): the Schur complement -C - B A^{-1}
    B^T, times omega^2 rho, acts on the Neumann modes as lap - omega^2/Vp^2
    (2-D and 3-D)."""
    lam, rho, om = 4.0, 1.5, 3.0
    S = const_system(n, h, lam, 0.0, rho, 0.0, om)
    Ainv = sp.diags(1.0 / sp.block_diag(S.A).diagonal())
    Schur = -S.C - S.B @ Ainv @ S.Bt
    for k in modes:
        v = cos_mode(n, k)
        ev = lap_eig(n, h, k) - om ** 2 * rho / lam
        np.testing.assert_allclose(om ** 2 * rho * (Schur @ v), ev * v, atol=1e-10 * (abs(ev) + 1))


def smooth_solution():
    import sympy as sy
    x, z = sy.symbols("x z")
    mu = 1 + sy.Rational(3, 10) * sy.sin(x + 2 * z)
    lam = 2 + sy.Rational(1, 2) * sy.cos(2 * x - z)
    rho = 1 + sy.Rational(1, 5) * sy.sin(3 * x * z)
    om = sy.Integer(2)
    u1 = sy.sin(sy.pi * x) * sy.cos(sy.pi * z)
    u2 = sy.cos(sy.pi * x) * sy.sin(sy.pi * z)
    p = -(lam + mu) * (sy.diff(u1, x) + sy.diff(u2, z))
    # Eq. 2.5 first row: -div(mu grad u_k) - rho omega^2 u_k + d_k p  (gamma = 0)
    f1 = -sy.diff(mu * sy.diff(u1, x), x) - sy.diff(mu * sy.diff(u1, z), z) - rho * om ** 2 * u1 + sy.diff(p, x)
    f2 = -sy.diff(mu * sy.diff(u2, x), x) - sy.diff(mu * sy.diff(u2, z), z) - rho * om ** 2 * u2 + sy.diff(p, z)
    L = lambda e: sy.lambdify((x, z), e, "numpy")
    return dict(mu=L(mu), lam=L(lam), rho=L(rho), u1=L(u1), u2=L(u2), p=L(p), f1=L(f1), f2=L(f2), om=2.0)


@pytest.mark.slow
def test_manufactured_solution_second_order():
    """Eq. 2.5 discretised by Eq. 2.6 converges at second order: the discrete
    solution of H [u;p] = [f;0] with f from a smooth exact (u, p) (p = -(lambda+mu)
    div u, gamma = 0) approaches the exact one with error ratio ~4 per halving."""
    pytest.importorskip("sympy")
    m = smooth_solution()
    errs = []
    for nn in (16, 32, 64):
        h = 1.0 / nn
        xc = (np.arange(nn) + 0.5) * h
        xf = np.arange(1, nn) * h
        Xc, Zc = np.meshgrid(xc, xc)                 # shape (n2, n1)
        S = elastic.assemble((nn, nn), (h, h), m["lam"](Xc, Zc), m["mu"](Xc, Zc), m["rho"](Xc, Zc),
                             np.zeros((nn, nn)), m["om"])
        X1, Z1 = np.meshgrid(xf, xc)                 # u1 faces: x = i h, z = cell
        X2, Z2 = np.meshgrid(xc, xf)                 # u2 faces
        rhs = np.concatenate([m["f1"](X1, Z1).ravel(), m["f2"](X2, Z2).ravel(), np.zeros(nn * nn)])
        sol = spla.spsolve(sp.csc_matrix(S.H), rhs)
        ex = np.concatenate([m["u1"](X1, Z1).ravel(), m["u2"](X2, Z2).ravel(), m["p"](Xc, Zc).ravel()])
        nu = S.sizes[0] + S.sizes[1]
        errs.append((np.abs(sol[:nu] - ex[:nu]).max(), np.abs(sol[nu:] - ex[nu:]).max()))
    for (eu0, ep0), (eu1, ep1) in zip(errs[:-1], errs[1:]):
        assert 3.2 < eu0 / eu1 < 5.0, errs
        assert 3.0 < ep0 / ep1 < 5.5, errs


@pytest.mark.parametrize("n,h", [((9, 7), (0.2, 0.2)), ((6, 5, 4), (0.2, 0.2, 0.2))])
def test_interior_commutator_vanishes_constant_medium(n, h):
    """Footnote to Eq. 2.10 and Sec. 4 (homogeneous media): on a MAC grid with
    constant coefficients the commutator Xi = B A - A_p B is exactly zero
    (here on every row, with the boundary reading R1), in 2-D and 3-D."""
    S = const_system(n, h)
    X = S.commutator()
    scale = abs(S.B).max() * abs(S.Ablk).max()
    assert abs(X).max() < 1e-12 * scale


def test_commutator_scaling_const_table():
    """Table 1, Const column: with constant lambda, mu, rho the commutator comes
    only from the absorbing layer's mass term and drops by ~100 between G_s = 10
    and G_s = 100 (0.00383 -> 3.74e-5): Xi is proportional to omega^2."""
    g = GOLD["commutator_const"]
    vals = []
    for gs in (10, 100):
        n1, n2 = 200, 64
        h1, h2 = 16.0 / n1, 5.0 / n2
        om = 2 * math.pi * 1.0 / (gs * h1)
        shape = (n2, n1)
        S = elastic.assemble((n1, n2), (h1, h2), 16 * np.ones(shape), np.ones(shape), np.ones(shape),
                             W.abc_gamma(shape, 20, om), om)
        vals.append(np.abs(S.commutator().data).mean())
    ratio_paper = g["gs10"] / g["gs100"]
    assert abs(vals[0] / vals[1] / ratio_paper - 1.0) < 0.05


def test_nnz_match_flop_model():
    """Sec. 4.4.2 FLOP model: A_1, A_2, H_p and A_p are 5-diagonal, each row of
    B has 2+2 entries, and the corrected right-hand side B r_u - A_p r_p costs 9
    entries per cell (interior rows)."""
    fm = GOLD["flop_model"]
    p = W.random_medium((10, 9), 7)
    S = elastic.from_problem(p)

    def interior_rows(M, n1, n2, off1=0, off2=0):
        M = sp.csr_matrix(M)
        nnz = np.diff(M.indptr).reshape(n2 - off2, n1 - off1)
        return nnz[2:-2, 2:-2]
    assert np.all(interior_rows(S.A[0], 10, 9, 1, 0) == fm["nnz_block_row"])
    assert np.all(interior_rows(S.A[1], 10, 9, 0, 1) == fm["nnz_block_row"])
    assert np.all(interior_rows(S.Hp, 10, 9) == fm["nnz_block_row"])
    assert np.all(interior_rows(S.Ap, 10, 9) == fm["nnz_block_row"])
    assert np.all(interior_rows(S.B, 10, 9) == fm["nnz_B_row"])
    assert fm["nnz_B_row"] + fm["nnz_block_row"] == fm["corrected_rhs_per_cell"]


@pytest.mark.parametrize("n", [(5, 4, 6)])
def test_3d_blocks_closed_form(n):
    """3-D version of Eq. 2.6: A_3 of a constant medium acts on
    cos(x1) cos(x2) sin(x3) modes with eigenvalue mu*lap - omega^2 rho~."""
    h = (0.3, 0.25, 0.2)
    lam, mu, rho, gam, om = 3.0, 1.5, 1.2, 0.7, 5.0
    S = const_system(n, h, lam, mu, rho, gam, om)
    rt = rho * (1 - 1j * gam / om)
    k = (2, 1, 3)
    v = np.einsum("k,j,i->kji", np.sin(math.pi * k[2] * np.arange(1, n[2]) / n[2]),
                  np.cos(math.pi * k[1] * (np.arange(n[1]) + 0.5) / n[1]),
                  np.cos(math.pi * k[0] * (np.arange(n[0]) + 0.5) / n[0])).ravel()
    ev = mu * lap_eig(n, h, k) - om ** 2 * rt
    np.testing.assert_allclose(S.A[2] @ v, ev * v, atol=1e-11 * abs(ev))
    assert abs(S.commutator()).max() < 1e-12 * abs(S.B).max() * abs(S.Ablk).max()
