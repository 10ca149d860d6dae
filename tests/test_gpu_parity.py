"""GPU parity: every step of the CUDA path, called through the C ABI, against
the FP64 CPU oracle on the same seeded inputs.

Tolerances (relative 2-norm errors):
  * operator apply H x (FP64 kernels vs FP64 sparse matrix): 1e-12, FP64
    rounding over a 19-entry row;
  * Galerkin stencils (FP64 setup kernels vs sparse R A P): 1e-12;
  * FP64-mode multigrid cycle / preconditioner: 1e-10 (same arithmetic, only
    the summation order differs; the coarse inverse can amplify rounding by
    its condition number, a few hundred here);
  * mixed-mode cycle / preconditioner: 2e-4.  Both sides use the identical
    bfloat16-rounded coefficients; the GPU computes in FP32 (unit roundoff
    6e-8) through about 20 dependent sweeps and restrictions and one coarse
    solve whose condition number (<= ~1e3 with the shift) amplifies the
    rounding of its right-hand side: 6e-8 * 20 * 1e3 ~ 1e-3 worst case, 2e-4
    with the observed cancellation margin of the random-phase inputs used;
  * solves: the true relative residual ||b - H x|| / ||b|| recomputed with the
    oracle's assembled H must be <= 1e-6 (the stopping rule of Sec. 4);
    FP64-mode iterates after a fixed number of steps agree with the oracle's
    FGMRES iterates to 1e-8.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import elastic, fgmres, multigrid as mg, precond

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_2411_15897_gb300 as bah  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def to_dev(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda")


def components(v, n):
    """Split a compact 2-D vector [u1 | u2 | p] into its three staggered
    lattices as arrays (u1: n2 x (n1-1), u2: (n2-1) x n1, p: n2 x n1)."""
    n1, n2 = n
    shapes = [(n2, n1 - 1), (n2 - 1, n1), (n2, n1)]
    out, o = [], 0
    for sh in shapes:
        k = sh[0] * sh[1]
        out.append(np.asarray(v[o:o + k]).reshape(sh))
        o += k
    return out


def check_elementwise(got, ref, n, tol):
    """Element by element, per staggered lattice: max |got - ref| <= tol *
    max |ref| over the whole lattice and over its boundary rows and columns
    alone (where the lattices differ).  A 2-norm check can hide one wrong row;
    this cannot."""
    for c, (g, r) in enumerate(zip(components(got, n), components(ref, n))):
        scale = np.abs(r).max()
        d = np.abs(g - r)
        assert d.max() <= tol * scale, (c, float(d.max() / scale))
        edge = max(d[0].max(), d[-1].max(), d[:, 0].max(), d[:, -1].max())
        assert edge <= tol * scale, (c, "boundary", float(edge / scale))


def to_host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_alpha(levels):
    return precond.default_alpha(levels)


PROBLEMS = {
    "random_48x40": lambda: W.random_medium((48, 40), 21, abc=4),
    "random_37x29": lambda: W.random_medium((37, 29), 22, abc=3),
    "layered_64x32": lambda: W.layered(64, 32, 4, seed=23, abc=6),
    "c1": lambda: W.config("c1"),
}


@pytest.fixture(scope="module")
def systems():
    return {}


def get(name, systems):
    if name not in systems:
        p = PROBLEMS[name]()
        systems[name] = (p, elastic.from_problem(p))
    return systems[name]


# ----------------------------------------------------------------------------
# operator apply (Eq. 2.6)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["random_48x40", "random_37x29", "c1"])
@pytest.mark.parametrize("conj", [0, 1])
def test_operator_apply_matches_oracle(name, conj, systems):
    p, S = get(name, systems)
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64, levels=1 if name == "random_37x29" else 0)
    x = W.random_vector(p.n, 5)
    y = to_host(s.apply_operator(to_dev(x), conj_transpose=bool(conj)))
    H = S.H.conj() if conj else S.H
    ref = H @ W.padded_to_compact(x, p.n)
    assert rel(W.padded_to_compact(y, p.n), ref) <= 1e-12
    # boundary-normal entries are written as zero and ignored on input
    pad = y.copy()
    pad_c = W.compact_to_padded(W.padded_to_compact(y, p.n), p.n)
    assert np.array_equal(pad, pad_c)
    x2 = x.copy()
    x2[0][:, 0] = 7.0 + 3.0j
    x2[1][0, :] = -2.0
    y2 = to_host(s.apply_operator(to_dev(x2), conj_transpose=bool(conj)))
    assert np.array_equal(y, y2)
    s.close()


def test_operator_apply_full_size_c2():
    """At the benchmark's size (512x512, layered), the whole output against the
    oracle's sparse matrix."""
    p = W.config("c2")
    S = elastic.from_problem(p)
    s = bah.Solver.from_problem(p, precision=bah.BAH_MIXED)
    x = W.random_vector(p.n, 9)
    y = to_host(s.apply_operator(to_dev(x)))
    assert rel(W.padded_to_compact(y, p.n), S.H @ W.padded_to_compact(x, p.n)) <= 1e-12
    s.close()


# ----------------------------------------------------------------------------
# Galerkin hierarchy (Eq. 4.3)
# ----------------------------------------------------------------------------
def stencil_to_matrix(st, rx, rz, kinds):
    """Compact sparse matrix from a padded slot-major stencil (test glue)."""
    ns, n2, n1 = st.shape
    valid = np.ones((n2, n1), bool)
    if kinds[0] == 'n':
        valid[:, 0] = False
    if kinds[1] == 'n':
        valid[0, :] = False
    idx = -np.ones((n2, n1), int)
    idx[valid] = np.arange(valid.sum())
    rows, cols, vals = [], [], []
    for dz in range(-rz, rz + 1):
        for dx in range(-rx, rx + 1):
            s = (dz + rz) * (2 * rx + 1) + (dx + rx)
            for j in range(n2):
                for i in range(n1):
                    if not valid[j, i]:
                        continue
                    jj, ii = j + dz, i + dx
                    if 0 <= jj < n2 and 0 <= ii < n1 and valid[jj, ii] and st[s, j, i] != 0:
                        rows.append(idx[j, i]); cols.append(idx[jj, ii]); vals.append(st[s, j, i])
    m = int(valid.sum())
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, m))


@pytest.mark.parametrize("intergrid", [0, 1])
def test_galerkin_stencils_match_oracle(intergrid, systems):
    p, S = get("layered_64x32", systems)
    levels = 3
    alpha = 0.3
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64, levels=levels, shift_alpha=alpha, intergrid=intergrid)
    blocks = [S.A_shifted(0, alpha), S.A_shifted(1, alpha), S.Hp_shifted(alpha)]
    for b in range(3):
        kinds = mg.block_kinds(2, b)
        hier = mg.build_hierarchy(blocks[b], p.n, kinds, levels, intergrid="mixed" if intergrid else "bilinear")
        for l in range(levels):
            st, rx, rz = bah.bah_level_stencil(s.ctx, b, l)
            M = stencil_to_matrix(st, rx, rz, kinds)
            ref = hier.ops_exact[l]
            assert abs(M - ref).max() <= 1e-12 * abs(ref).max(), (b, l)
    s.close()


# ----------------------------------------------------------------------------
# one multigrid cycle per block, and the preconditioner (Sec. 3, Sec. 4.4.1)
# ----------------------------------------------------------------------------
def block_vector(p, b, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)
    if b == 0:
        v[:, 0] = 0
    if b == 1:
        v[0, :] = 0
    return v


def block_compact(v, b):
    return (v[:, 1:] if b == 0 else (v[1:, :] if b == 1 else v)).ravel()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["layered_64x32", "random_48x40"])
def test_block_cycle_matches_oracle(prec, name, systems):
    p, S = get(name, systems)
    levels = 3
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64 if prec == "fp64" else bah.BAH_MIXED, levels=levels)
    alpha = precond.default_alpha(levels)
    pc = precond.multigrid(S, levels, alpha, precision=prec)
    tol = 1e-10 if prec == "fp64" else 2e-4
    for b in range(3):
        v = block_vector(p, b, 100 + b)
        x = to_host(s.block_cycle(b, to_dev(v)))
        ref = mg.cycle(pc.hier[b], block_compact(v, b))
        assert rel(block_compact(x, b), ref) <= tol, (b, rel(block_compact(x, b), ref))
        # structural zeros stay zero
        if b == 0:
            assert np.all(x[:, 0] == 0)
        if b == 1:
            assert np.all(x[0, :] == 0)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["layered_64x32", "random_48x40", "c1", "random_37x29"])
def test_preconditioner_matches_oracle(prec, name, systems):
    """z = P^{-1} D r against the oracle, as a 2-norm and element by element
    per lattice (boundary rows included), with the small levels in the
    shared-memory cluster kernel (mixed mode) and the staged Galerkin sweeps;
    37x29 is odd in both directions (a 1-level hierarchy)."""
    p, S = get(name, systems)
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64 if prec == "fp64" else bah.BAH_MIXED)
    pc = precond.multigrid(S, s.levels, precond.default_alpha(s.levels), precision=prec)
    r = W.random_vector(p.n, 31)
    z = to_host(s.apply_preconditioner(to_dev(r)))
    ref = pc.apply(W.padded_to_compact(r, p.n))
    zc = W.padded_to_compact(z, p.n)
    tol = 1e-10 if prec == "fp64" else 2e-4
    assert rel(zc, ref) <= tol
    check_elementwise(zc, ref, p.n, 1e-9 if prec == "fp64" else 2e-3)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nu", [(1, 3), (2, 3), (0, 3), (2, 2)])
def test_preconditioner_smoothing_counts_match_oracle(prec, nu, systems, monkeypatch):
    """V(nu1,nu2) cycles with other sweep counts (the benchmark runs V(1,3)):
    odd and even numbers of buffer swaps, a zero pre-smoothing count, on the
    separate kernels and with the small levels in the cluster kernel."""
    p, S = get("layered_64x32", systems)
    r = W.random_vector(p.n, 49)
    pc = precond.multigrid(S, 4, precond.default_alpha(4), precision=prec, nu_pre=nu[0], nu_post=nu[1])
    ref = pc.apply(W.padded_to_compact(r, p.n))
    tol = 1e-10 if prec == "fp64" else 2e-4
    for smem in ("0", "1"):
        monkeypatch.setenv("BAH_SMEM_MG", smem)
        s = bah.Solver.from_problem(p, precision=bah.BAH_FP64 if prec == "fp64" else bah.BAH_MIXED, levels=4,
                                    nu_pre=nu[0], nu_post=nu[1])
        z = to_host(s.apply_preconditioner(to_dev(r)))
        assert rel(W.padded_to_compact(z, p.n), ref) <= tol, (smem, rel(W.padded_to_compact(z, p.n), ref))
        s.close()


# ----------------------------------------------------------------------------
# solves
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("prec,krylov", [("fp64", 0), ("mixed", 0), ("fp64", 1), ("mixed", 1)])
def test_solve_c1_reaches_tolerance(prec, krylov, systems):
    p, S = get("c1", systems)
    s = bah.Solver.from_problem(p, precision=bah.BAH_FP64 if prec == "fp64" else bah.BAH_MIXED, krylov_arith=krylov)
    b = W.point_source(p)
    x, status, st = s.solve(to_dev(b), rtol=1e-6)
    assert status == bah.BAH_OK, st
    xc = W.padded_to_compact(to_host(x), p.n)
    bc = W.padded_to_compact(b, p.n)
    rr = np.linalg.norm(bc - S.H @ xc) / np.linalg.norm(bc)
    assert rr <= 1e-6
    assert abs(rr - st[0]["relres_true"]) <= 1e-9
    xs = spla.spsolve(sp.csc_matrix(S.H), bc)
    assert rel(xc, xs) <= 1e-3
    s.close()


@pytest.mark.parametrize("krylov", [bah.BAH_KRYLOV_FP64, bah.BAH_KRYLOV_DF])
def test_solve_fp64_iterates_match_oracle_fgmres(krylov, systems):
    """FP64 multigrid: the GPU's FGMRES(20) iterate after k steps equals the
    oracle's (same preconditioner, same Krylov space; selective
    reorthogonalisation vs MGS), with the Krylov basis in FP64 or in
    double-FP32 (48-bit) arithmetic."""
    p, S = get("layered_64x32", systems)
    for k in (3, 7, 25):
        s = bah.Solver.from_problem(p, precision=bah.BAH_FP64, maxit=k, levels=3, krylov_arith=krylov)
        b = W.point_source(p)
        x, status, st = s.solve(to_dev(b), rtol=1e-12)
        pc = precond.multigrid(S, 3, precond.default_alpha(3))
        H = S.H
        ref = fgmres.fgmres(lambda v: H @ v, W.padded_to_compact(b, p.n), pc.apply, restart=20, rtol=1e-12, maxit=k)
        assert st[0]["iters"] == ref.iters == k
        assert rel(W.padded_to_compact(to_host(x), p.n), ref.x) <= 1e-8
        s.close()


@pytest.mark.parametrize("krylov", [bah.BAH_KRYLOV_FP64, bah.BAH_KRYLOV_DF])
def test_solve_c2_full_size_mixed_and_host_buffers(krylov):
    """The benchmark workload (512x512 layered) in the launch configuration the
    benchmark times: mixed precision, default options; the residual is
    recomputed by the oracle's assembled operator.  The same solve through host
    buffers gives the same iterate."""
    p = W.config("c2")
    S = elastic.from_problem(p)
    s = bah.Solver.from_problem(p, precision=bah.BAH_MIXED, krylov_arith=krylov)
    b = W.point_source(p)
    x, status, st = s.solve(to_dev(b), rtol=1e-6)
    assert status == bah.BAH_OK, st
    xc = W.padded_to_compact(to_host(x), p.n)
    bc = W.padded_to_compact(b, p.n)
    assert np.linalg.norm(bc - S.H @ xc) / np.linalg.norm(bc) <= 1e-6
    # the Arnoldi estimate tracks the true residual: the operator inside FGMRES
    # is accurate far below the tolerance
    assert abs(st[0]["relres_est"] - st[0]["relres_true"]) <= 1e-3 * st[0]["relres_true"], st[0]
    xh, status_h, st_h = s.solve(b.copy(), rtol=1e-6)
    assert status_h == bah.BAH_OK and st_h[0]["iters"] == st[0]["iters"]
    assert rel(W.padded_to_compact(xh, p.n), xc) <= 1e-12
    s.close()


def test_preconditioner_full_size_c2_matches_oracle():
    """The benchmark's preconditioner at full size (512x512 layered, default
    options: 6 levels, shift 1.0, levels 2-5 in the cluster kernel, staged
    Galerkin sweeps on level 1) against the oracle's mixed-precision
    preconditioner, element by element over the whole vector."""
    p = W.config("c2")
    S = elastic.from_problem(p)
    s = bah.Solver.from_problem(p)
    assert s.levels == 6 and s.info["cluster_level"] == 2
    r = W.random_vector(p.n, 47)
    z = to_host(s.apply_preconditioner(to_dev(r)))
    pc = precond.multigrid(S, 6, precond.default_alpha(6), precision="mixed")
    zc, ref = W.padded_to_compact(z, p.n), pc.apply(W.padded_to_compact(r, p.n))
    assert rel(zc, ref) <= 2e-4
    check_elementwise(zc, ref, p.n, 2e-3)
    s.close()


# ----------------------------------------------------------------------------
# edge cases and error behaviour
# ----------------------------------------------------------------------------
def test_zero_rhs_and_empty_batch(systems):
    p, S = get("random_48x40", systems)
    s = bah.Solver.from_problem(p)
    b = torch.zeros(s.shape, dtype=torch.complex128, device="cuda")
    x, status, st = s.solve(b)
    assert status == bah.BAH_OK and st[0]["iters"] == 0
    assert torch.count_nonzero(x).item() == 0
    out = torch.zeros(1, dtype=torch.complex128, device="cuda")
    assert bah.bah_apply_operator(s.ctx, out, out, 0) == bah.BAH_OK
    s.close()


def test_invalid_arguments_are_reported():
    p = W.random_medium((16, 16), 1)
    with pytest.raises(bah.BahError) as e:
        bah.Solver(p.n, p.h, p.lam, p.mu, p.rho, p.gamma, -1.0)
    assert e.value.status == bah.BAH_ERR_ARG
    with pytest.raises(bah.BahError) as e:
        bah.Solver(p.n, p.h, p.lam, p.mu, p.rho, p.gamma, p.omega, restart=0)
    assert e.value.status == bah.BAH_ERR_ARG
    with pytest.raises(bah.BahError) as e:
        bah.Solver(p.n, p.h, p.lam, p.mu, p.rho, p.gamma, p.omega, levels=6)
    assert e.value.status == bah.BAH_ERR_ARG


def test_not_converged_status(systems):
    p, S = get("c1", systems)
    s = bah.Solver.from_problem(p, maxit=3)
    x, status, st = s.solve(to_dev(W.point_source(p)))
    assert status == bah.BAH_ERR_NOT_CONVERGED and st[0]["iters"] == 3
    assert st[0]["relres_true"] > 1e-6
    s.close()


def test_multiple_rhs_sequential(systems):
    p, S = get("random_48x40", systems)
    s = bah.Solver.from_problem(p)
    b = np.stack([W.random_vector(p.n, 40 + k) for k in range(3)])
    x, status, st = s.solve(to_dev(b), rtol=1e-8)
    assert status == bah.BAH_OK
    xh = to_host(x)
    for k in range(3):
        bc = W.padded_to_compact(b[k], p.n)
        xc = W.padded_to_compact(xh[k], p.n)
        assert np.linalg.norm(bc - S.H @ xc) / np.linalg.norm(bc) <= 1e-8
    s.close()


def test_graph_and_direct_launch_paths_agree(systems, monkeypatch):
    """The per-step CUDA graphs replay exactly the kernels of the direct launch
    path: identical iterates, bit for bit."""
    p, S = get("random_48x40", systems)
    b = to_dev(W.point_source(p))
    s1 = bah.Solver.from_problem(p, maxit=30)
    x1, _, st1 = s1.solve(b)
    monkeypatch.setenv("BAH_NO_GRAPHS", "1")
    s2 = bah.Solver.from_problem(p, maxit=30)
    x2, _, st2 = s2.solve(b)
    assert st1[0]["iters"] == st2[0]["iters"]
    assert torch.equal(x1, x2)
    s1.close()
    s2.close()


@pytest.mark.parametrize("cls", ["jacobi", "residual", "dot"])
def test_profile_counters(cls, systems):
    """Launch and byte counters advance and timed classes report device time."""
    p, S = get("c1", systems)
    s = bah.Solver.from_problem(p, maxit=5)
    bah.bah_profile_control(s.ctx, 1 << bah.BAH_K_NAMES.index(cls), True)
    s.solve(to_dev(W.point_source(p)))
    pr = bah.bah_profile_read(s.ctx)
    assert pr["launches"] > 5 * 10
    assert pr["classes"][cls]["ms"] > 0 and pr["classes"][cls]["bytes"] > 0
    other = "axpy" if cls == "dot" else "dot"
    assert pr["classes"][other]["ms"] == 0
    s.close()


@pytest.mark.parametrize("cycle", [bah.BAH_CYCLE_V, bah.BAH_CYCLE_W])
@pytest.mark.parametrize("levels", [4, 5])
def test_smem_cluster_multigrid_matches_separate_kernels(cycle, levels, monkeypatch):
    """Mixed mode holds the small levels (from the first one that fits, down
    to the coarsest) in one cluster's shared memory.  Against the separate
    kernels (BAH_SMEM_MG=0): the same preconditioner to FP32 rounding, V and
    W cycles, slabs that leave some CTAs without rows (8x4 and 16x8 levels on
    a 16-CTA cluster); against the oracle to the mixed-mode tolerance; and
    batched solves (5 sources in batches of 2) with identical counts."""
    p = W.layered(128, 64, 5, seed=29, abc=8)
    S = elastic.from_problem(p)
    r = W.random_vector(p.n, 41)
    cyc = "W" if cycle == bah.BAH_CYCLE_W else "V"
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("BAH_SMEM_MG", mode)
        s = bah.Solver.from_problem(p, levels=levels, cycle=cycle)
        if mode == "1":
            bah.bah_profile_control(s.ctx, 0, True)
        out[mode] = to_host(s.apply_preconditioner(to_dev(r)))
        if mode == "1":
            pr = bah.bah_profile_read(s.ctx)
            assert pr["classes"]["cluster"]["calls"] >= 2, pr["classes"]["cluster"]
            assert pr["classes"]["coarse"]["calls"] == 0
        s.close()
    assert rel(out["1"], out["0"]) <= 1e-6, rel(out["1"], out["0"])
    pc = precond.multigrid(S, levels, precond.default_alpha(levels), precision="mixed", cycle=cyc)
    assert rel(W.padded_to_compact(out["1"], p.n), pc.apply(W.padded_to_compact(r, p.n))) <= 2e-4
    b = np.stack([W.point_source(p, (12 + 24 * k, 8)) for k in range(5)])
    xs = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("BAH_SMEM_MG", mode)
        s = bah.Solver.from_problem(p, levels=levels, cycle=cycle, rhs_block=2, maxit=20000)
        x, st, stats = s.solve(to_dev(b), rtol=1e-7)
        assert st == bah.BAH_OK
        xs[mode] = (to_host(x), [q["iters"] for q in stats])
        s.close()
    assert xs["0"][1] == xs["1"][1]
    assert rel(xs["1"][0], xs["0"][0]) <= 1e-5
    xh = xs["1"][0]
    for k in range(5):
        bc = W.padded_to_compact(b[k], p.n)
        assert np.linalg.norm(bc - S.H @ W.padded_to_compact(xh[k], p.n)) / np.linalg.norm(bc) <= 1e-7


@pytest.mark.parametrize("name", ["random_48x40", "layered_64x32"])
def test_staged_level_kernels_match_plain(name, systems, monkeypatch):
    """Mixed mode stages each CTA's stencil coefficients and iterate rows in
    shared memory before a Jacobi sweep or residual on a Galerkin level; with
    BAH_STAGED=0 the plain kernels read them directly.  Same arithmetic:
    identical preconditioner (to rounding), and equal to the oracle's."""
    p, S = get(name, systems)
    r = W.random_vector(p.n, 45)
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("BAH_STAGED", mode)
        monkeypatch.setenv("BAH_SMEM_MG", "0")     # keep every level on the separate kernels
        s = bah.Solver.from_problem(p, levels=3)
        out[mode] = to_host(s.apply_preconditioner(to_dev(r)))
        s.close()
    assert rel(out["1"], out["0"]) <= 1e-6, rel(out["1"], out["0"])
    pc = precond.multigrid(S, 3, precond.default_alpha(3), precision="mixed")
    assert rel(W.padded_to_compact(out["1"], p.n), pc.apply(W.padded_to_compact(r, p.n))) <= 2e-4


def test_double_float_operator_in_fgmres(monkeypatch):
    """In mixed mode with the double-float basis, w = H z is formed in
    double-float arithmetic (about 2^-47 relative).  An operator that is only
    FP32-accurate would make the Arnoldi residual estimate drift from the true
    residual by ~1e-7 relative to ||b||, i.e. ~10% at convergence; here the two
    agree to 1e-3 relative, the iteration count equals the FP64-operator
    run's to within 2, and the true residual (recomputed by the oracle's
    assembled operator) meets the tolerance."""
    p = W.layered(128, 64, 5, seed=29, abc=8)
    S = elastic.from_problem(p)
    b = W.point_source(p)
    bc = W.padded_to_compact(b, p.n)
    res = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("BAH_OP_F64", mode)
        s = bah.Solver.from_problem(p, krylov_arith=bah.BAH_KRYLOV_DF, maxit=20000)
        x, status, st = s.solve(to_dev(b), rtol=1e-7)
        assert status == bah.BAH_OK, st
        xc = W.padded_to_compact(to_host(x), p.n)
        rr = np.linalg.norm(bc - S.H @ xc) / np.linalg.norm(bc)
        assert rr <= 1e-7
        res[mode] = st[0]
        s.close()
    q = res["0"]
    assert abs(q["relres_est"] - q["relres_true"]) <= 1e-3 * q["relres_true"], q
    assert abs(res["0"]["iters"] - res["1"]["iters"]) <= 2, res


# ----------------------------------------------------------------------------
# batched right-hand sides
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("prec,krylov", [(bah.BAH_MIXED, 0), (bah.BAH_FP64, 0), (bah.BAH_MIXED, 1)])
def test_batched_solve_equals_sequential(prec, krylov, systems):
    """rhs_block > 1 advances independent FGMRES recurrences in lockstep with
    the same per-right-hand-side arithmetic: identical iterates and counts,
    including a ragged last batch (5 right-hand sides, batches of 3)."""
    p, S = get("layered_64x32", systems)
    srcs = [(8 + 12 * k, 6) for k in range(5)]
    b = np.stack([W.point_source(p, s) for s in srcs])
    s1 = bah.Solver.from_problem(p, precision=prec, levels=3, krylov_arith=krylov)
    x1, st1, stats1 = s1.solve(to_dev(b), rtol=1e-7)
    s3 = bah.Solver.from_problem(p, precision=prec, levels=3, rhs_block=3, krylov_arith=krylov)
    x3, st3, stats3 = s3.solve(to_dev(b), rtol=1e-7)
    assert st1 == st3 == bah.BAH_OK
    assert [q["iters"] for q in stats1] == [q["iters"] for q in stats3]
    assert rel(to_host(x3), to_host(x1)) <= 1e-13
    xh = to_host(x3)
    for k in range(len(srcs)):
        bc = W.padded_to_compact(b[k], p.n)
        assert np.linalg.norm(bc - S.H @ W.padded_to_compact(xh[k], p.n)) / np.linalg.norm(bc) <= 1e-7
    s1.close()
    s3.close()


def test_batched_multisource_layered():
    """A C4-shaped problem at reduced size: 8 sources along the top row of a
    layered 128x64 medium, solved in one batch; every residual recomputed by
    the oracle's operator.  (The oracle itself needs 3900-4500 FGMRES(20)
    iterations on this medium, hence the raised iteration limit.)"""
    p = W.layered(128, 64, 6, seed=5, abc=8, nsrc=8, src_spacing=16)
    S = elastic.from_problem(p)
    b = W.all_sources(p)
    s = bah.Solver.from_problem(p, rhs_block=8, maxit=15000)
    x, status, stats = s.solve(to_dev(b), rtol=1e-6)
    assert status == bah.BAH_OK
    xh = to_host(x)
    for k in range(8):
        bc = W.padded_to_compact(b[k], p.n)
        assert np.linalg.norm(bc - S.H @ W.padded_to_compact(xh[k], p.n)) / np.linalg.norm(bc) <= 1e-6
        assert stats[k]["relres_true"] <= 1e-6
    s.close()
