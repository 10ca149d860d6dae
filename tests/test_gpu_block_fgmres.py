"""GPU block FGMRES (block_krylov = 1: one Krylov space for a batch of
right-hand sides; block Arnoldi with two passes of block classical
Gram-Schmidt and CholQR2) against the oracle's block FGMRES.

* FP64 mode, the same multigrid preconditioner on both sides: after k block
  steps the GPU iterates equal the oracle's to 1e-8 (the same block Krylov
  space and the same minimisation; only the summation order differs).
* Mixed mode, eight sources of a layered medium: every column reaches 1e-6 by
  the oracle's assembled operator, in no more block iterations than the
  slowest source needs in the lockstep (independent) form.
"""
import numpy as np
import pytest

import workloads as W
from oracle import block_fgmres as BF
from oracle import elastic, precond

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_2411_15897_gb300 as bah  # noqa: E402


def to_dev(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda")


@pytest.mark.parametrize("s", [2, 4, 5])
def test_block_fgmres_iterates_match_oracle(s):
    p = W.layered(64, 32, 4, seed=23, abc=6, nsrc=s, src_spacing=10)
    S = elastic.from_problem(p)
    B = np.stack([W.point_source(p, q) for q in p.sources])
    Bc = np.column_stack([W.padded_to_compact(B[k], p.n) for k in range(s)])
    pc = precond.multigrid(S, 3, precond.default_alpha(3))
    Mb = lambda V: np.column_stack([pc.apply(V[:, c]) for c in range(V.shape[1])])
    for k in (2, 5, 12):
        ref = BF.block_fgmres(lambda V: S.H @ V, Bc, Mb, restart=10, rtol=1e-14, maxit=k)
        sv = bah.Solver.from_problem(p, precision=bah.BAH_FP64, levels=3, restart=10, maxit=k, rhs_block=s,
                                     block_krylov=1)
        x, status, st = sv.solve(to_dev(B), rtol=1e-14)
        torch.cuda.synchronize()
        X = x.cpu().numpy()
        assert all(q["iters"] == k for q in st), [q["iters"] for q in st]
        for c in range(s):
            got = W.padded_to_compact(X[c], p.n)
            err = np.linalg.norm(got - ref.X[:, c]) / np.linalg.norm(ref.X[:, c])
            assert err <= 1e-8, (k, c, err)
        sv.close()


def test_block_fgmres_mixed_converges_and_needs_no_more_steps_than_lockstep():
    p = W.layered(256, 128, 5, seed=31, abc=10, nsrc=8, src_spacing=24)
    S = elastic.from_problem(p)
    B = np.stack([W.point_source(p, q) for q in p.sources])
    lock = bah.Solver.from_problem(p, rhs_block=8, restart=10, maxit=20000)
    _, st_l, stats_l = lock.solve(to_dev(B), rtol=1e-6)
    lock.close()
    assert st_l == bah.BAH_OK
    blk = bah.Solver.from_problem(p, rhs_block=8, restart=10, maxit=20000, block_krylov=1)
    x, st_b, stats_b = blk.solve(to_dev(B), rtol=1e-6)
    assert st_b == bah.BAH_OK, stats_b
    torch.cuda.synchronize()
    X = x.cpu().numpy()
    for c in range(8):
        bc = W.padded_to_compact(B[c], p.n)
        rr = np.linalg.norm(bc - S.H @ W.padded_to_compact(X[c], p.n)) / np.linalg.norm(bc)
        assert rr <= 1e-6 * (1 + 1e-9), (c, rr)
    its_lock = max(q["iters"] for q in stats_l)
    print(f"block FGMRES: {stats_b[0]['iters']} block iterations; lockstep: max {its_lock}")
    assert stats_b[0]["iters"] <= its_lock
    blk.close()


def test_block_fgmres_option_checks():
    p = W.layered(64, 32, 4, seed=23, abc=6)
    with pytest.raises(bah.BahError) as e:
        bah.Solver.from_problem(p, rhs_block=1, block_krylov=1)
    assert e.value.status == bah.BAH_ERR_UNSUPPORTED
    with pytest.raises(bah.BahError) as e:
        bah.Solver.from_problem(p, rhs_block=4, block_krylov=1, krylov_arith=bah.BAH_KRYLOV_DF)
    assert e.value.status == bah.BAH_ERR_UNSUPPORTED
