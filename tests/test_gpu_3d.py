"""GPU parity on 3-D grids, through the C ABI: the operator (Eq. 2.6), the four
acoustic block cycles with the mixed intergrid of Eq. 4.4 (the paper's 3-D
multigrid, Sec. 4.5: W(2,2) with Jacobi weights 0.8, 0.8, 0.2; V(1,2) as well),
the block-acoustic preconditioner (Eq. 3.3 - 3.5) and full solves, against the
FP64 CPU oracle on the same seeded inputs.

Tolerances (relative 2-norm errors):
  * operator apply: 1e-12 (FP64 on both sides, at most 13 entries per row);
  * FP64-mode cycles and preconditioner: 1e-10 (the same arithmetic in another
    summation order, amplified at most by the coarsest inverse's condition
    number, a few hundred here);
  * mixed-mode cycles and preconditioner: 2e-4, against the oracle's
    mixed-precision preconditioner, which rounds every level's stencil below
    the coarsest to bfloat16 as the GPU stores it (the 3-D distributor keeps
    FP64 coefficients on both sides); the GPU then computes in
    FP32 (unit roundoff 6e-8) through about 20 dependent sweeps and the
    coarsest solve, whose condition number (<= ~1e3) amplifies the rounding of
    its right-hand side, as in 2-D;
  * solves: the true relative residual ||b - H x|| / ||b|| recomputed with the
    oracle's assembled H must be <= 1e-6 (the stopping rule of Sec. 4), and
    FP64-mode iterates after a fixed number of FGMRES steps equal the oracle's
    FGMRES iterates to 1e-8.
"""
import numpy as np
import pytest

import workloads as W
from oracle import elastic, fgmres, multigrid as mg, precond

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_2411_15897_gb300 as bah  # noqa: E402

# cycle settings on the library side and the same on the oracle side
CYCLES = {
    "W22": (dict(cycle=bah.BAH_CYCLE_W, nu_pre=2, nu_post=2, jacobi_w=(0.8, 0.8, 0.2)),
            dict(cycle="W", nu_pre=2, nu_post=2, weights=(0.8, 0.8, 0.2))),
    "V12": (dict(cycle=bah.BAH_CYCLE_V, nu_pre=1, nu_post=2, jacobi_w=(0.8, 0.8, 0.3)),
            dict(cycle="V", nu_pre=1, nu_post=2, weights=(0.8, 0.8, 0.3))),
}
W22 = CYCLES["W22"][0]
C5_ALPHA = 0.4
PREC = {"fp64": bah.BAH_FP64, "mixed": bah.BAH_MIXED}
TOL = {"fp64": 1e-10, "mixed": 2e-4}


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def to_dev(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda")


def to_host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def solver(p, prec="fp64", **kw):
    return bah.Solver.from_problem(p, precision=PREC[prec], intergrid=bah.BAH_INTERGRID_MIXED, **kw)


_CACHE = {}


def small():
    """Rough random medium on 16 x 12 x 8 cells, anisotropic spacing."""
    if "small" not in _CACHE:
        p = W.random_medium((16, 12, 8), 52, abc=2, h=(1 / 16, 1 / 14, 1 / 18))
        _CACHE["small"] = (p, elastic.from_problem(p))
    return _CACHE["small"]


def block_vector(n, q, seed):
    rng = np.random.default_rng(seed)
    shp = tuple(reversed(n))
    v = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    if q < 3:
        sl = [slice(None)] * 3
        sl[2 - q] = 0
        v[tuple(sl)] = 0
    return v


def block_compact(v, q):
    if q == 3:
        return v.ravel()
    sl = [slice(None)] * 3
    sl[2 - q] = slice(1, None)
    return v[tuple(sl)].ravel()


# ----------------------------------------------------------------------------
# operator apply (Eq. 2.6)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("conj", [0, 1])
def test_3d_operator_apply_matches_oracle(conj):
    p = W.random_medium((10, 8, 6), 51, abc=2, h=(0.1, 0.125, 1 / 12))
    S = elastic.from_problem(p)
    s = solver(p)
    x = W.random_vector(p.n, 5)
    y = to_host(s.apply_operator(to_dev(x), conj_transpose=bool(conj)))
    H = S.H.conj() if conj else S.H
    assert rel(W.padded_to_compact(y, p.n), H @ W.padded_to_compact(x, p.n)) <= 1e-12
    # boundary-normal entries are written as zero and ignored on input
    assert np.array_equal(y, W.compact_to_padded(W.padded_to_compact(y, p.n), p.n))
    x2 = x.copy()
    x2[0][:, :, 0] = 7.0 + 3.0j
    x2[1][:, 0, :] = -2.0
    x2[2][0, :, :] = 5.0j
    y2 = to_host(s.apply_operator(to_dev(x2), conj_transpose=bool(conj)))
    assert np.array_equal(y, y2)
    s.close()


# ----------------------------------------------------------------------------
# one cycle per block, and the preconditioner
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cyc", ["V12", "W22"])
def test_3d_block_cycle_matches_oracle(prec, cyc):
    p, S = small()
    levels = 3
    alpha = precond.default_alpha(levels)
    s = solver(p, prec, levels=levels, shift_alpha=alpha, **CYCLES[cyc][0])
    pc = precond.multigrid(S, levels, alpha, intergrid="mixed", precision=prec, **CYCLES[cyc][1])
    for q in range(4):
        v = block_vector(p.n, q, 200 + q)
        x = to_host(s.block_cycle(q, to_dev(v)))
        ref = mg.cycle(pc.hier[q], block_compact(v, q))
        assert rel(block_compact(x, q), ref) <= TOL[prec], (q, rel(block_compact(x, q), ref))
        if q < 3:
            sl = [slice(None)] * 3
            sl[2 - q] = 0
            assert np.all(x[tuple(sl)] == 0)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nu", [(1, 2), (2, 2), (0, 3)])
def test_3d_preconditioner_matches_oracle(prec, nu):
    """Default hierarchy of the 16 x 12 x 8 grid (coarsest at most 256 cells),
    V(nu1, nu2): odd and even numbers of buffer swaps and a zero pre-smoothing
    count."""
    p, S = small()
    s = solver(p, prec, nu_pre=nu[0], nu_post=nu[1])
    pc = precond.multigrid(S, s.levels, s.alpha, intergrid="mixed", nu_pre=nu[0], nu_post=nu[1], precision=prec,
                           bf16_ap=False)
    r = W.random_vector(p.n, 31)
    z = to_host(s.apply_preconditioner(to_dev(r)))
    assert rel(W.padded_to_compact(z, p.n), pc.apply(W.padded_to_compact(r, p.n))) <= TOL[prec]
    s.close()


# ----------------------------------------------------------------------------
# solves
# ----------------------------------------------------------------------------
def test_3d_solve_fp64_iterates_match_oracle_fgmres():
    """FP64 mode, W(2,2): after k FGMRES(20) steps the GPU iterate equals the
    oracle's (same preconditioner and Krylov space; selective
    reorthogonalisation against MGS)."""
    p, S = small()
    b = W.point_source(p)
    pc = precond.multigrid(S, 3, 0.2, intergrid="mixed", **CYCLES["W22"][1])
    for k in (4, 23):
        s = solver(p, "fp64", levels=3, shift_alpha=0.2, maxit=k, **W22)
        x, status, st = s.solve(to_dev(b), rtol=1e-12)
        ref = fgmres.fgmres(lambda v: S.H @ v, W.padded_to_compact(b, p.n), pc.apply, restart=20, rtol=1e-12,
                            maxit=k)
        assert st[0]["iters"] == ref.iters == k
        assert rel(W.padded_to_compact(to_host(x), p.n), ref.x) <= 1e-8
        s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_3d_solve_batches_reach_tolerance(prec):
    """Three point sources in batches of two (the last batch holds one) reach
    the tolerance, each checked with the oracle's assembled H."""
    p, S = small()
    srcs = [(8, 6, 2), (3, 9, 4), (12, 2, 6)]
    b = np.stack([W.point_source(p, s) for s in srcs])
    s = solver(p, prec, rhs_block=2, **W22)
    x, status, st = s.solve(to_dev(b), rtol=1e-6)
    assert status == bah.BAH_OK, st
    xh = to_host(x)
    for k in range(3):
        bc = W.padded_to_compact(b[k], p.n)
        rr = np.linalg.norm(bc - S.H @ W.padded_to_compact(xh[k], p.n)) / np.linalg.norm(bc)
        assert rr <= 1e-6, (k, rr)
        assert abs(rr - st[k]["relres_true"]) <= 1e-9
    s.close()


def test_3d_c5_full_size_mixed():
    """The 128^3 random-field workload (8 points per shear wavelength, 10-cell
    absorbing layer, top-face point source): mixed precision, W(2,2) with the
    mixed intergrid on 5 levels (coarsest 8^3), FGMRES(20) to 1e-6; the true
    residual is recomputed with the oracle's assembled H at full size."""
    p = W.config("c5")
    S = elastic.from_problem(p)
    free0, _ = torch.cuda.mem_get_info()
    s = solver(p, "mixed", levels=5, shift_alpha=C5_ALPHA, maxit=3000, **W22)
    free1, _ = torch.cuda.mem_get_info()
    b = W.point_source(p)
    x, status, st = s.solve(to_dev(b), rtol=1e-6)
    assert status == bah.BAH_OK, st
    bc = W.padded_to_compact(b, p.n)
    rr = np.linalg.norm(bc - S.H @ W.padded_to_compact(to_host(x), p.n)) / np.linalg.norm(bc)
    assert rr <= 1e-6
    assert abs(rr - st[0]["relres_true"]) <= 1e-9
    print(f"c5: {st[0]['iters']} iterations, context {(free0 - free1) / 2**30:.2f} GiB")
    s.close()


def test_3d_unsupported_requests_are_reported():
    p, S = small()
    s = solver(p)
    g = np.zeros(p.lam.size)
    x = to_dev(W.random_vector(p.n, 3))
    with pytest.raises(bah.BahError) as e:
        bah.bah_gradient(s.ctx, x, x, 1, to_dev(g), to_dev(g), to_dev(g))
    assert e.value.status == bah.BAH_ERR_UNSUPPORTED
    with pytest.raises(bah.BahError) as e:
        bah.bah_level_stencil(s.ctx, 0, 0)
    assert e.value.status == bah.BAH_ERR_UNSUPPORTED
    s.close()
