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
