"""Pins of the oracle's 3-D path (the paper's 3-D experiments, Sec. 4.5: mixed
intergrid, W(2,2) cycles) against what the paper and the mathematics fix
(no GPU)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import elastic, multigrid as mg, precond

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def fine_sizes(n, kinds):
    return [n[a] - 1 if kinds[a] == 'n' else n[a] for a in range(3)]


def coarse_sizes(n, kinds):
    return [n[a] // 2 - 1 if kinds[a] == 'n' else n[a] // 2 for a in range(3)]


def unflatten(idx, sizes):
    """Compact index -> per-axis compact coordinates (x_1 fastest)."""
    return idx % sizes[0], (idx // sizes[0]) % sizes[1], idx // (sizes[0] * sizes[1])


@pytest.mark.parametrize("block", [0, 1, 2, 3])
def test_3d_mixed_restriction_rows_are_printed_stencils(block):
    """Eq. 4.4 in 3-D: an interior row of the mixed restriction is the
    Kronecker product of 1/4[1 2 1] along the block's nodal axis and 1/2[1 * 1]
    along its cell-centred axes."""
    st = GOLD["restriction_stencils"]
    n = (8, 10, 12)
    kinds = mg.block_kinds(3, block)
    _, R = mg.transfers(n, kinds, "mixed")
    m, mc = fine_sizes(n, kinds), coarse_sizes(n, kinds)
    J = (1, 2, 3)                                   # interior coarse point, compact coordinates
    row = R.getrow((J[2] * mc[1] + J[1]) * mc[0] + J[0]).toarray().reshape(m[2], m[1], m[0])

    def one(a):
        if kinds[a] == 'n':                          # coarse face K = J+1 sits on fine face 2K
            K = J[a] + 1
            return [2 * K - 2 + t for t in range(3)], st["nodal"]
        return [2 * J[a] + t for t in range(2)], st["cell_mixed"]
    (ix, wx), (iy, wy), (iz, wz) = one(0), one(1), one(2)
    exp = np.zeros_like(row)
    for c, z in zip(iz, wz):
        for b, y in zip(iy, wy):
            for a, x in zip(ix, wx):
                exp[c, b, a] = x * y * z
    np.testing.assert_array_equal(row, exp)
    # every row of the mixed restriction sums to one (boundary rows included)
    np.testing.assert_allclose(R @ np.ones(R.shape[1]), 1.0, atol=1e-14)


@pytest.mark.parametrize("block", [0, 1, 2, 3])
def test_3d_prolongation_exact_on_linear_functions(block):
    """Trilinear prolongation reproduces a linear function at every fine point
    not adjacent to the boundary (samples at the staggered locations)."""
    n = (8, 10, 12)
    kinds = mg.block_kinds(3, block)
    P, _ = mg.transfers(n, kinds, "mixed")
    h = [1.0 / v for v in n]

    def coords(nn, kind, hh):
        return np.arange(1, nn) * hh if kind == 'n' else (np.arange(nn) + 0.5) * hh
    f = lambda x, y, z: 0.3 + 1.7 * x - 0.9 * y + 0.6 * z
    cf = [coords(n[a], kinds[a], h[a]) for a in range(3)]
    cc = [coords(n[a] // 2, kinds[a], 2 * h[a]) for a in range(3)]
    Zc, Yc, Xc = np.meshgrid(cc[2], cc[1], cc[0], indexing="ij")
    Zf, Yf, Xf = np.meshgrid(cf[2], cf[1], cf[0], indexing="ij")
    fine = (P @ f(Xc, Yc, Zc).ravel()).reshape(Xf.shape)
    np.testing.assert_allclose(fine[1:-1, 1:-1, 1:-1], f(Xf, Yf, Zf)[1:-1, 1:-1, 1:-1], atol=1e-13)


@pytest.mark.parametrize("block", [0, 1, 2, 3])
def test_3d_galerkin_width(block):
    """Galerkin coarsening (Eq. 4.3) of a 7-point block: with the mixed
    intergrid every coarse row couples only to coarse points within one cell
    per axis (a 27-point stencil, which the 3-D GPU levels store), while the
    bilinear restriction widens every cell-centred axis to two cells."""
    n = (8, 8, 8)
    p = W.random_medium(n, 61, abc=1)
    S = elastic.from_problem(p)
    A = (S.A_shifted(block, 0.3) if block < 3 else S.Hp_shifted(0.3)).tocsr()
    kinds = mg.block_kinds(3, block)
    mc = coarse_sizes(n, kinds)
    for intergrid, widths in (("mixed", [1, 1, 1]), ("bilinear", [1 if k == 'n' else 2 for k in kinds])):
        P, R = mg.transfers(n, kinds, intergrid)
        Ac = sp.coo_matrix(R @ A @ P)
        Ac.eliminate_zeros()
        rc, cc = np.array(unflatten(Ac.row, mc)), np.array(unflatten(Ac.col, mc))
        reach = np.abs(rc - cc).max(axis=1)
        assert list(reach) == widths, (intergrid, list(reach))


def test_3d_two_grid_exact_coarse_is_projection():
    """Algorithm 1 without relaxation and with an exact coarse solve has error
    propagation I - P (R A P)^{-1} R A, a projection, for the mixed intergrid
    too (R is not a multiple of P^T there)."""
    n = (8, 8, 8)
    p = W.random_medium(n, 62, abc=1)
    S = elastic.from_problem(p)
    A = S.Hp_shifted(0.3).toarray()
    P, R = mg.transfers(n, ['c', 'c', 'c'], "mixed")
    P, R = P.toarray(), R.toarray()
    E = np.eye(A.shape[0]) - P @ np.linalg.solve(R @ A @ P, R @ A)
    np.testing.assert_allclose(E @ E, E, atol=1e-10)
    h = mg.build_hierarchy(sp.csr_matrix(A), n, ['c', 'c', 'c'], 2, nu_pre=0, nu_post=0, intergrid="mixed")
    b = np.random.default_rng(0).standard_normal(A.shape[0]) + 0j
    np.testing.assert_allclose(mg.cycle(h, b), P @ np.linalg.solve(R @ A @ P, R @ b), atol=1e-12)


def test_3d_theorem1_spectrum():
    """Theorem 1 in 3-D: P^{-1} K has the eigenvalue 1 with multiplicity at
    least the size of A (three displacement blocks), and
    spec(I - P^{-1} K) = spec(Z) u {0}, Z = Xi A^{-1} B^T H_p^{-1}."""
    p = W.random_medium((4, 4, 3), 9, omega=4.0, abc=1)
    S = elastic.from_problem(p)
    Pm, D, K = precond.dense_matrices(S, 0.0)
    nA = sum(S.sizes[:3])
    T = np.eye(Pm.shape[0]) - np.linalg.solve(Pm, K)
    eT = np.linalg.eigvals(T)
    scale = max(1.0, np.abs(eT).max())
    assert np.sum(np.abs(eT) < 1e-7 * scale) >= nA
    A = sp.block_diag(S.A).toarray()
    Z = S.commutator().toarray() @ np.linalg.solve(A, S.Bt.toarray()) @ np.linalg.inv(S.Hp.toarray())
    eZ = np.linalg.eigvals(Z)
    nzT = np.sort_complex(eT[np.abs(eT) >= 1e-7 * scale])
    nzZ = np.sort_complex(eZ[np.abs(eZ) >= 1e-7 * scale])
    assert len(nzT) == len(nzZ)
    np.testing.assert_allclose(nzT, nzZ, atol=1e-6 * scale)


def test_3d_w22_cycle_is_a_contraction():
    """The paper's 3-D cycle (W(2,2), Jacobi 0.8/0.8/0.2, mixed intergrid) on a
    shifted displacement block is a convergent stationary iteration."""
    n = (16, 16, 16)
    p = W.random_medium(n, 63, abc=2)
    S = elastic.from_problem(p)
    A = S.A_shifted(2, 0.5)
    h = mg.build_hierarchy(A, n, mg.block_kinds(3, 2), 3, weights=(0.8, 0.8, 0.2), nu_pre=2, nu_post=2,
                           cycle="W", intergrid="mixed")
    rng = np.random.default_rng(5)
    b = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    x = np.zeros_like(b)
    res = []
    for _ in range(6):
        x = x + mg.cycle(h, b - A @ x)
        res.append(np.linalg.norm(b - A @ x))
    assert res[-1] / res[0] < 0.5 ** 5


def _smooth_solution_3d():
    import sympy as sy
    x, y, z = sy.symbols("x y z")
    mu = 1 + sy.Rational(3, 10) * sy.sin(x + 2 * y - z)
    lam = 2 + sy.Rational(1, 2) * sy.cos(2 * x - y + z)
    rho = 1 + sy.Rational(1, 5) * sy.sin(3 * x * z + y)
    om = sy.Integer(2)
    X = (x, y, z)
    # normal displacement zero on every face; tangential derivatives vanish there too
    u = [sy.sin(sy.pi * x) * sy.cos(sy.pi * y) * sy.cos(sy.pi * z),
         sy.cos(sy.pi * x) * sy.sin(sy.pi * y) * sy.cos(sy.pi * z),
         sy.cos(sy.pi * x) * sy.cos(sy.pi * y) * sy.sin(sy.pi * z)]
    p = -(lam + mu) * sum(sy.diff(u[k], X[k]) for k in range(3))
    # Eq. 2.5 first row per component: -div(mu grad u_k) - rho omega^2 u_k + d_k p  (gamma = 0)
    f = [-sum(sy.diff(mu * sy.diff(u[k], X[j]), X[j]) for j in range(3)) - rho * om ** 2 * u[k] + sy.diff(p, X[k])
         for k in range(3)]
    L = lambda e: sy.lambdify(X, e, "numpy")
    return dict(mu=L(mu), lam=L(lam), rho=L(rho), u=[L(e) for e in u], p=L(p), f=[L(e) for e in f], om=2.0)


NN_3D = (16, 32, 64)


def test_3d_manufactured_truncation_second_order():
    """Eq. 2.5 discretised by Eq. 2.6 in 3-D is consistent at second order: for a
    smooth exact (u, p) with p = -(lambda+mu) div u and gamma = 0 on variable
    lambda, mu, rho, the truncation error H [u; p] - [f; 0] at points two
    cells inside the domain falls by ~4 per halving of h (a dropped term, a
    wrong sign or a misplaced average leaves an O(1) error).  Measured ratios
    on 16, 32, 64 cells per axis: 3.4 and 3.9 (u), 3.0 and 3.7 (p)."""
    pytest.importorskip("sympy")
    m = _smooth_solution_3d()
    errs = []
    for nn in NN_3D:
        h = 1.0 / nn
        c = (np.arange(nn) + 0.5) * h
        fc = np.arange(1, nn) * h
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        S = elastic.assemble((nn, nn, nn), (h, h, h), m["lam"](X, Y, Z), m["mu"](X, Y, Z), m["rho"](X, Y, Z),
                             np.zeros((nn, nn, nn)), m["om"])
        ex, rhs, keep = [], [], []
        for k in range(3):
            ax = [c, c, c]
            ax[k] = fc
            Zk, Yk, Xk = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
            ex.append(m["u"][k](Xk, Yk, Zk).ravel())
            rhs.append(m["f"][k](Xk, Yk, Zk).ravel())
            idx = np.meshgrid(*[np.arange(len(ax[a])) for a in (2, 1, 0)], indexing="ij")
            keep.append(np.all([(q >= 2) & (q <= len(ax[a]) - 3) for q, a in zip(idx, (2, 1, 0))], axis=0).ravel())
        ex.append(m["p"](X, Y, Z).ravel())
        rhs.append(np.zeros(nn ** 3))
        idx = np.meshgrid(*[np.arange(nn)] * 3, indexing="ij")
        keep.append(np.all([(q >= 2) & (q <= nn - 3) for q in idx], axis=0).ravel())
        tau = S.H @ np.concatenate(ex) - np.concatenate(rhs)
        tau, keep = np.abs(tau), np.concatenate(keep)
        nu = sum(S.sizes[:3])
        errs.append((tau[:nu][keep[:nu]].max(), tau[nu:][keep[nu:]].max()))
    ratios = [(eu0 / eu1, ep0 / ep1) for (eu0, ep0), (eu1, ep1) in zip(errs[:-1], errs[1:])]
    for ru, rp in ratios:
        assert 2.8 < ru < 4.8 and 2.8 < rp < 4.8, (errs, ratios)
    # the finest pair is close to the asymptotic factor 4
    assert 3.5 < ratios[-1][0] < 4.5 and 3.5 < ratios[-1][1] < 4.5, (errs, ratios)
