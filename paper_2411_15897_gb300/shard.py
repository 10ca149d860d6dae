"""Host-side logic for running the solver on several GPUs, one process each.

Point sources are independent solves (the right-hand sides of H x_s = b_s,
Eq. 2.6), so a job over many sources is split by source: rank r of N takes
sources r, r + N, r + 2N, ...  No data crosses between ranks during the
solves. A misfit gradient summed over sources (see ``misfit.py``) needs one
sum of the three cell fields and the scalar misfit at the end, which
``sum_over_ranks`` does. Timing is reported as the maximum over ranks.

Only ``torch.distributed`` collectives are used; with one process (no
initialised process group) every function is the identity.
"""
from __future__ import annotations

import numpy as np


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def rank_and_world():
    d = _dist()
    return (d.get_rank(), d.get_world_size()) if d else (0, 1)


def shard(n_sources: int, rank: int, world: int) -> np.ndarray:
    """Indices of the sources that rank ``rank`` of ``world`` solves (strided, so
    neighbouring sources, which converge alike, spread over the ranks)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    return np.arange(rank, n_sources, world, dtype=np.int64)


def max_over_ranks(value: float, device="cpu") -> float:
    """Largest value over all ranks (the job's time is the slowest rank's)."""
    d = _dist()
    if d is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(*tensors):
    """In-place sum over all ranks of each tensor (gradient fields, misfit);
    returns the tensors."""
    d = _dist()
    if d is not None:
        for t in tensors:
            d.all_reduce(t, op=d.ReduceOp.SUM)
    return tensors
