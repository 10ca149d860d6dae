"""GPU adjoint gradient (a torch.autograd.Function over the C ABI) against the
CPU oracle's adjoint gradient and central finite differences."""
import numpy as np
import pytest

import workloads as W
from oracle import elastic, gradient as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_2411_15897_gb300 as bah  # noqa: E402
from paper_2411_15897_gb300 import misfit as M  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def problem(n=(16, 12), seed=3, nsrc=2, row=2):
    p = W.random_medium(n, seed, abc=2)
    srcs = [(3 + 6 * k, 5) for k in range(nsrc)]
    B = np.stack([W.point_source(p, s) for s in srcs])
    rec = M.receiver_indices(p.n, row)
    rng = np.random.default_rng(seed + 100)
    St = elastic.assemble(p.n, p.h, p.lam * (1 + 0.1 * rng.standard_normal(p.shape)),
                          p.mu * (1 + 0.1 * rng.standard_normal(p.shape)),
                          p.rho * (1 + 0.05 * rng.standard_normal(p.shape)), p.gamma, p.omega)
    Bc = np.column_stack([W.padded_to_compact(B[k], p.n) for k in range(nsrc)])
    rows = G.receiver_rows(St, [(i, row) for i in range(p.n[0])])
    D = G.forward(St, Bc)[rows, :]
    return p, B, Bc, rec, rows, D


def test_gradient_kernel_matches_oracle_definition():
    """bah_gradient on the oracle's own forward and adjoint fields equals the
    oracle's -Re y^H (dH/dm_k) x with dH/dm_k assembled per cell (1e-12)."""
    p, B, Bc, rec, rows, D = problem()
    S = elastic.from_problem(p)
    J, g, X, Y = G.gradient(S, Bc, D, rows)
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64)
    Xp = np.stack([W.compact_to_padded(X[:, k], p.n) for k in range(X.shape[1])])
    Yp = np.stack([W.compact_to_padded(Y[:, k], p.n) for k in range(Y.shape[1])])
    gd = torch.zeros(3, S.ncells, dtype=torch.float64, device="cuda")
    bah.bah_gradient(s.ctx, torch.from_numpy(Xp).cuda(), torch.from_numpy(Yp).cuda(), X.shape[1], gd[0], gd[1], gd[2])
    torch.cuda.synchronize()
    gh = gd.cpu().numpy()
    for i, prm in enumerate(("lambda", "mu", "rho")):
        assert rel(gh[i], g[prm]) <= 1e-12, prm
    s.close()


def test_misfit_adjoint_source_and_adjoint_solve():
    p, B, Bc, rec, rows, D = problem()
    S = elastic.from_problem(p)
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64, rhs_block=2)
    b = torch.from_numpy(B).cuda()
    x = torch.zeros_like(b)
    st, _ = bah.bah_solve(s.ctx, b, x, 2, 1e-12)
    Dd = torch.from_numpy(np.ascontiguousarray(D.T)).cuda()
    adj = torch.empty_like(b)
    mis = torch.empty(2, dtype=torch.float64, device="cuda")
    r = torch.from_numpy(rec).cuda()
    bah.bah_misfit(s.ctx, x, Dd, r, rec.size, 2, adj, mis)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    for k in range(2):
        xc = W.padded_to_compact(xh[k], p.n)
        resid = xc[rows] - D[:, k]
        assert abs(mis[k].item() - 0.5 * np.sum(np.abs(resid) ** 2)) <= 1e-9 * mis[k].item()
        ac = W.padded_to_compact(adj[k].cpu().numpy(), p.n)
        assert np.allclose(ac[rows], resid, rtol=1e-12, atol=0) and np.count_nonzero(ac) == rows.size
    # adjoint solve: H^H y = adj
    y = torch.zeros_like(adj)
    st, stats = bah.bah_solve_adjoint(s.ctx, adj, y, 2, 1e-10)
    assert st == bah.BAH_OK
    yh = y.cpu().numpy()
    HH = S.H.conj().T
    for k in range(2):
        ac = W.padded_to_compact(adj[k].cpu().numpy(), p.n)
        yc = W.padded_to_compact(yh[k], p.n)
        assert np.linalg.norm(ac - HH @ yc) / np.linalg.norm(ac) <= 1e-10
    s.close()


def test_misfit_repeated_receivers_sum():
    """A receiver index listed twice (with different data) enters the misfit
    twice and the adjoint source as the sum of both residuals: Q^H (Q x - d)
    as the oracle forms it (np.add.at), to 1e-13."""
    p, B, Bc, rec, rows, D = problem()
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64, rhs_block=2)
    rec2 = np.concatenate([rec, rec[3:6], rec[4:5]]).astype(np.int32)
    rows2 = np.concatenate([rows, rows[3:6], rows[4:5]])
    D2 = np.concatenate([D, D[3:6] * (1 + 0.3j), D[4:5] * (0.5 - 1j)])
    xh = np.stack([W.random_vector(p.n, 70 + k) for k in range(2)])
    x = torch.from_numpy(xh).cuda()
    Dd = torch.from_numpy(np.ascontiguousarray(D2.T)).cuda()
    adj = torch.empty_like(x)
    mis = torch.empty(2, dtype=torch.float64, device="cuda")
    bah.bah_misfit(s.ctx, x, Dd, torch.from_numpy(rec2).cuda(), rec2.size, 2, adj, mis)
    torch.cuda.synchronize()
    for k in range(2):
        xc = W.padded_to_compact(xh[k], p.n)
        resid = xc[rows2] - D2[:, k]
        ref = np.zeros_like(xc)
        np.add.at(ref, rows2, resid)
        assert abs(mis[k].item() - 0.5 * np.sum(np.abs(resid) ** 2)) <= 1e-12 * mis[k].item()
        ac = W.padded_to_compact(adj[k].cpu().numpy(), p.n)
        assert np.abs(ac - ref).max() <= 1e-13 * np.abs(ref).max()
    s.close()


def _J(p, lam, mu, rho, b, d, r, rtol=1e-11):
    return M.misfit(lam, mu, rho, p.gamma, p.omega, p.n, p.h, b, d, r,
                    dict(precision=bah.BAH_FP64, rhs_block=2), rtol)


def test_autograd_gradient_matches_oracle_and_central_differences():
    """torch.autograd through ReceiverMisfit: the gradient w.r.t. lambda, mu,
    rho matches the oracle's adjoint gradient (direct solves) and central
    finite differences of the GPU misfit on 16 random cells (FP64 solves to
    rel-res 1e-11)."""
    p, B, Bc, rec, rows, D = problem()
    S = elastic.from_problem(p)
    J0, g, _, _ = G.gradient(S, Bc, D, rows)
    b = torch.from_numpy(B).cuda()
    d = torch.from_numpy(np.ascontiguousarray(D.T)).cuda()
    r = torch.from_numpy(rec).cuda()
    lam = torch.tensor(p.lam, dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(p.mu, dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(p.rho, dtype=torch.float64, requires_grad=True)
    J = _J(p, lam, mu, rho, b, d, r)
    assert abs(J.item() - J0) <= 1e-8 * J0
    J.backward()
    grads = {"lambda": lam.grad.numpy().ravel(), "mu": mu.grad.numpy().ravel(), "rho": rho.grad.numpy().ravel()}
    for prm in grads:
        assert rel(grads[prm], g[prm]) <= 1e-7, prm
    rng = np.random.default_rng(6)
    cells = rng.choice(S.ncells, 16, replace=False)
    for prm, base in (("lambda", p.lam), ("mu", p.mu), ("rho", p.rho)):
        for k in cells:
            m0 = base.ravel()[k]
            eps = 1e-5 * abs(m0)
            vals = []
            for sgn in (1, -1):
                arrs = {"lambda": p.lam.copy(), "mu": p.mu.copy(), "rho": p.rho.copy()}
                arrs[prm].ravel()[k] = m0 + sgn * eps
                with torch.no_grad():
                    vals.append(_J(p, *(torch.tensor(arrs[q]) for q in ("lambda", "mu", "rho")), b, d, r).item())
            fd = (vals[0] - vals[1]) / (2 * eps)
            scale = max(abs(fd), 1e-3 * np.abs(grads[prm]).max())
            assert abs(fd - grads[prm][k]) <= 1e-4 * scale, (prm, k, fd, grads[prm][k])
