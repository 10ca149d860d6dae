"""The several-GPU path's host logic on CPU: two processes joined by a gloo
process group (no GPU).  Sources are split across ranks with no exchange
during the solves; the job's time is the maximum over ranks; a misfit
gradient over all sources is the sum over ranks of each rank's gradient over
its own sources.  The per-rank gradient here is the oracle's (adjoint state
with sparse direct solves), so the test checks the decomposition, not the
GPU kernels."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2411_15897_gb300 import shard  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def problem(nsrc=5):
    import workloads as W
    from oracle import elastic, gradient as G
    p = W.random_medium((10, 8), 3, abc=2)
    S = elastic.from_problem(p)
    srcs = [(1 + 2 * k, 3) for k in range(nsrc)]
    B = np.column_stack([W.padded_to_compact(W.point_source(p, s), p.n) for s in srcs])
    rows = G.receiver_rows(S, [(i, 2) for i in range(p.n[0])])
    rng = np.random.default_rng(7)
    St = elastic.assemble(p.n, p.h, p.lam * (1 + 0.1 * rng.standard_normal(p.shape)), p.mu, p.rho, p.gamma,
                          p.omega)
    D = G.forward(St, B)[rows, :]
    return S, B, D, rows


def worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import gradient as G
        assert shard.rank_and_world() == (rank, world)
        # timing: the maximum over ranks
        assert shard.max_over_ranks(10.0 + rank) == 10.0 + world - 1
        # gradient over this rank's sources, summed over ranks
        S, B, D, rows = problem()
        mine = shard.shard(B.shape[1], rank, world)
        J, g, _, _ = G.gradient(S, B[:, mine], D[:, mine], rows)
        tens = [torch.tensor(g[k]) for k in ("lambda", "mu", "rho")] + [torch.tensor([J], dtype=torch.float64)]
        shard.sum_over_ranks(*tens)
        if rank == 0:
            np.savez(out, lam=tens[0].numpy(), mu=tens[1].numpy(), rho=tens[2].numpy(), J=tens[3].numpy(),
                     mine=mine)
    finally:
        dist.destroy_process_group()


def test_shard_covers_every_source_once():
    for n in (1, 5, 64):
        for world in (1, 2, 3, 8):
            parts = [shard.shard(n, r, world) for r in range(world)]
            allidx = np.sort(np.concatenate(parts))
            assert np.array_equal(allidx, np.arange(n))
    with pytest.raises(ValueError):
        shard.shard(4, 2, 2)


def test_single_process_is_identity():
    assert shard.rank_and_world() == (0, 1)
    assert shard.max_over_ranks(3.5) == 3.5
    t = torch.ones(3)
    shard.sum_over_ranks(t)
    assert torch.equal(t, torch.ones(3))


def test_two_ranks_gloo_gradient_and_timing(tmp_path):
    """world_size 2 over gloo: the summed per-rank gradients equal the gradient
    over all sources in one process (to rounding), and max-over-ranks timing."""
    out = str(tmp_path / "rank0.npz")
    mp.spawn(worker, args=(2, free_port(), out), nprocs=2, join=True)
    from oracle import gradient as G
    S, B, D, rows = problem()
    J, g, _, _ = G.gradient(S, B, D, rows)
    r = np.load(out)
    assert np.array_equal(r["mine"], np.array([0, 2, 4]))
    assert abs(r["J"][0] - J) <= 1e-12 * abs(J)
    for k, key in (("lambda", "lam"), ("mu", "mu"), ("rho", "rho")):
        assert np.linalg.norm(r[key] - g[k]) <= 1e-12 * np.linalg.norm(g[k])
