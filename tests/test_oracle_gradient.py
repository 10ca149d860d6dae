"""Pins of the oracle's adjoint gradient (no GPU): central finite differences
of the misfit with direct solves, and the adjoint identity."""
import numpy as np
import pytest

import workloads as W
from oracle import elastic, gradient as G


def setup(n=(10, 8), seed=3, nsrc=2):
    p = W.random_medium(n, seed, abc=2 if len(n) == 2 else 1)
    S = elastic.from_problem(p)
    if len(n) == 2:
        srcs = [(2 + 4 * k, 3) for k in range(nsrc)]
        rec = [(i, 2) for i in range(n[0])]
    else:                      # sources and a receiver plane on the u_3 faces at x_3-index 2
        srcs = [(1 + 2 * k, 2, 3) for k in range(nsrc)]
        rec = [(i, j, 2) for j in range(n[1]) for i in range(n[0])]
    B = np.column_stack([W.padded_to_compact(W.point_source(p, s), p.n) for s in srcs])
    rows = G.receiver_rows(S, rec)
    # observed data from a perturbed ("true") medium
    rng = np.random.default_rng(seed + 100)
    St = elastic.assemble(p.n, p.h, p.lam * (1 + 0.1 * rng.standard_normal(p.shape)),
                          p.mu * (1 + 0.1 * rng.standard_normal(p.shape)),
                          p.rho * (1 + 0.05 * rng.standard_normal(p.shape)), p.gamma, p.omega)
    D = G.forward(St, B)[rows, :]
    return p, S, B, D, rows


def J_at(p, field, k, value, B, D, rows):
    arrs = {"lambda": p.lam.copy(), "mu": p.mu.copy(), "rho": p.rho.copy()}
    arrs[field].ravel()[k] = value
    S = elastic.assemble(p.n, p.h, arrs["lambda"], arrs["mu"], arrs["rho"], p.gamma, p.omega)
    return G.misfit(S, B, D, rows)[0]


def test_receiver_rows_pick_the_u_d_component():
    p, S, B, D, rows = setup()
    sizes = S.sizes
    assert np.all(rows >= sizes[0]) and np.all(rows < sizes[0] + sizes[1])
    pad = np.zeros(W.padded_shape(p.n), complex)
    pad[1][2, 3] = 1.0       # u2 face (i=3, j=2)
    c = W.padded_to_compact(pad, p.n)
    assert np.flatnonzero(c)[0] == G.receiver_rows(S, [(3, 2)])[0]


@pytest.mark.parametrize("n", [(10, 8), (5, 4, 4)])
@pytest.mark.parametrize("field", ["lambda", "mu", "rho"])
def test_adjoint_gradient_matches_central_differences(field, n):
    """dJ/dm_k by the adjoint state equals the central difference of J with
    exact (sparse direct) solves, on random cells of a 10x8 (2-D) and a
    5x4x4 (3-D, three displacement blocks and edge means per axis pair)
    random medium."""
    p, S, B, D, rows = setup(n)
    J0, g, X, Y = G.gradient(S, B, D, rows, params=(field,))
    rng = np.random.default_rng(11)
    for k in rng.choice(S.ncells, 6, replace=False):
        m0 = {"lambda": p.lam, "mu": p.mu, "rho": p.rho}[field].ravel()[k]
        eps = 1e-5 * abs(m0)
        fd = (J_at(p, field, k, m0 + eps, B, D, rows) - J_at(p, field, k, m0 - eps, B, D, rows)) / (2 * eps)
        assert abs(fd - g[field][k]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g[field]).max()), (k, fd, g[field][k])


def test_adjoint_identity_conjugate_transpose():
    """<H x, y> = <x, H^H y> with H^H = conj(H) (H complex symmetric)."""
    p, S, B, D, rows = setup()
    rng = np.random.default_rng(2)
    x = rng.standard_normal(S.H.shape[0]) + 1j * rng.standard_normal(S.H.shape[0])
    y = rng.standard_normal(S.H.shape[0]) + 1j * rng.standard_normal(S.H.shape[0])
    lhs = np.vdot(y, S.H @ x)
    rhs = np.vdot(S.H.conj() @ y, x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_repeated_receiver_counts_twice_in_the_adjoint_source():
    """Q with a repeated row (a receiver listed twice) weighs that datum twice
    in J, so Q^H (Q x - d) must sum both copies: the adjoint gradient still
    equals the central difference of J."""
    p, S, B, D, rows = setup()
    rows2 = np.concatenate([rows, rows[3:5]])
    D2 = np.concatenate([D, D[3:5] * (1 + 0.3j)])
    J0, g, X, Y = G.gradient(S, B, D2, rows2, params=("mu",))
    rng = np.random.default_rng(13)
    for k in rng.choice(S.ncells, 4, replace=False):
        m0 = p.mu.ravel()[k]
        eps = 1e-5 * abs(m0)
        fd = (J_at(p, "mu", k, m0 + eps, B, D2, rows2) - J_at(p, "mu", k, m0 - eps, B, D2, rows2)) / (2 * eps)
        assert abs(fd - g["mu"][k]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g["mu"]).max()), (k, fd, g["mu"][k])
