"""The allocation-free relative-residual entry point.

bah_residual_norm_static serves callers that cannot call cudaMalloc when they
need the residual (real-time loops that forbid allocator calls after start-up,
because an allocation can block for an unbounded time, or hosts whose device
memory all belongs to another allocator): its reduction scratch is a static
device array instead of context workspace.  Checked through the C ABI against the relative residual that
bah_solve reports for the same b and x, and against the CPU oracle, on two
calls in a row (the static array keeps the previous call's contents).
This file sorts last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

import workloads as W
from oracle import elastic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_2411_15897_gb300 as bah  # noqa: E402


def test_static_residual_matches_solver_and_oracle():
    p = W.random_medium((48, 40), 21, abc=4)
    S = elastic.from_problem(p)
    s = bah.Solver.from_problem(p)
    nrhs = 3
    bh = np.stack([W.point_source(p)] + [W.random_vector(p.n, 70 + k) for k in range(nrhs - 1)])
    b = torch.from_numpy(bh).cuda()
    x, status, st = s.solve(b, rtol=1e-8)
    assert status == bah.BAH_OK
    xr = torch.from_numpy(np.stack([W.random_vector(p.n, 90 + k) for k in range(nrhs)])).cuda()
    out = torch.empty(nrhs, dtype=torch.float64, device="cuda")
    for call in range(2):
        # converged iterates: against the residual bah_solve reported
        out.fill_(-1.0)
        bah.bah_residual_norm_static(s.ctx, b, x, nrhs, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for k in range(nrhs):
            ref = st[k]["relres_true"]
            assert abs(got[k] - ref) <= 1e-9 * ref, (call, k, got[k], ref)
        # arbitrary iterates: against the oracle's assembled operator
        out.fill_(-1.0)
        bah.bah_residual_norm_static(s.ctx, b, xr, nrhs, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        xh = xr.cpu().numpy()
        for k in range(nrhs):
            bc = W.padded_to_compact(bh[k], p.n)
            ref = np.linalg.norm(bc - S.H @ W.padded_to_compact(xh[k], p.n)) / np.linalg.norm(bc)
            assert abs(got[k] - ref) <= 1e-12 * ref, (call, k, got[k], ref)
    # sizes beyond the static scratch are rejected with a clear error
    big = bah.BAH_STATIC_MAX_RHS + 1
    with pytest.raises(bah.BahError) as e:
        bah.bah_residual_norm_static(s.ctx, b, x, big, out)
    assert e.value.status == bah.BAH_ERR_ARG and "BAH_STATIC_MAX_RHS" in bah.last_error()
    s.close()


def test_static_residual_rejects_3d_contexts():
    """The entry point covers 2-D grids only: a 3-D context is refused with
    BAH_ERR_UNSUPPORTED before anything is launched."""
    p = W.random_medium((8, 8, 8), 52, abc=1)
    s = bah.Solver.from_problem(p, intergrid=bah.BAH_INTERGRID_MIXED, levels=2)
    n = int(np.prod(W.padded_shape(p.n)))
    b = torch.zeros(n, dtype=torch.complex128, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(bah.BahError) as e:
        bah.bah_residual_norm_static(s.ctx, b, b, 1, out)
    assert e.value.status == bah.BAH_ERR_UNSUPPORTED
    s.close()
