"""Autotuner for batched solves: how many right-hand sides one batch holds
(``rhs_block``) and which multigrid launch variant runs, chosen by timing
short solves on the device.

Point sources are independent solves of H x_s = b_s (Eq. 2.6).  A batch of s
sources advances s FGMRES recurrences in lockstep: every multigrid, operator
and Gram-Schmidt launch covers the whole batch, so a larger batch amortises
launches and coefficient reads over more sources, until the batch's vectors
no longer fit the caches and each launch becomes bandwidth-bound.  Where that
turns over depends on the grid and the device, so it is measured: each
candidate runs a fixed number of FGMRES iterations on its batch (tolerance
below reach, so no source stops early) and the cost per source and iteration
is compared.  The variants are the library's per-context launch switches
(environment variables read when a context is created): the shared-memory
cluster multigrid of the small levels (``BAH_SMEM_MG``) and the
shared-memory staging of the Galerkin-level sweeps (``BAH_STAGED``).

Results are cached in a JSON file keyed by grid, sources, precision and
device, so a job tunes once.  ``tune`` takes the timing function as an
argument; the default one runs on the current CUDA device.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

# launch variants: name -> environment settings at context creation
VARIANTS = {
    "default": {},
    "no-cluster-mg": {"BAH_SMEM_MG": "0"},
    "no-staging": {"BAH_STAGED": "0"},
}


@dataclass
class Choice:
    rhs_block: int
    variant: str
    cost: float                       # seconds per source per FGMRES iteration
    table: dict = field(default_factory=dict)   # "rhs_block/variant" -> cost

    def as_dict(self):
        return {"rhs_block": self.rhs_block, "variant": self.variant, "cost": self.cost, "table": self.table}


def _key(problem, nsrc, opts, device):
    prec = opts.get("precision", "default")
    return f"{'x'.join(map(str, problem.n))}|{nsrc}|{prec}|{device}"


def time_batch(problem, rhs_block, env, opts, iters):
    """Seconds per source per FGMRES iteration for one batch of ``rhs_block``
    sources of ``problem`` run for exactly ``iters`` iterations on the current
    CUDA device (one untimed run, then one timed by CUDA events)."""
    import numpy as np
    import torch

    import workloads as W
    from . import Solver, bah_solve

    saved = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        s = Solver.from_problem(problem, **dict(opts, rhs_block=rhs_block, maxit=iters))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    srcs = [problem.sources[i % len(problem.sources)] for i in range(rhs_block)]
    b = torch.from_numpy(np.stack([W.point_source(problem, q) for q in srcs])).cuda()
    x = torch.zeros_like(b)
    bah_solve(s.ctx, b, x, rhs_block, 1e-30)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    bah_solve(s.ctx, b, x, rhs_block, 1e-30)
    e1.record(stream)
    e1.synchronize()
    s.close()
    return e0.elapsed_time(e1) * 1e-3 / (rhs_block * iters)


def candidates(nsrc, limit=256):
    """Powers of two up to the number of sources (and the library's limit),
    plus the number of sources itself."""
    out, b = [], 1
    while b <= min(nsrc, limit):
        out.append(b)
        b *= 2
    if nsrc <= limit and nsrc not in out:
        out.append(nsrc)
    return out


def tune(problem, nsrc=None, opts=None, iters=20, variants=None, measure=time_batch, cache_path=None,
         device=None) -> Choice:
    """Cheapest (rhs_block, variant) per source and iteration for ``nsrc``
    sources of ``problem``.  ``measure(problem, rhs_block, env, opts, iters)``
    returns seconds per source per iteration; ``cache_path`` (JSON) stores
    the choice under the problem's key and is read back on the next call."""
    opts = dict(opts or {})
    nsrc = int(nsrc or len(problem.sources) or 1)
    variants = variants or VARIANTS
    if device is None:
        try:
            import torch
            device = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
        except Exception:
            device = "unknown"
    key = _key(problem, nsrc, opts, device)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            c = cache[key]
            return Choice(c["rhs_block"], c["variant"], c["cost"], c.get("table", {}))
    table = {}
    best = None
    for rb in candidates(nsrc):
        for name, env in variants.items():
            cost = float(measure(problem, rb, env, opts, iters))
            table[f"{rb}/{name}"] = cost
            if best is None or cost < best.cost:
                best = Choice(rb, name, cost)
    best.table = table
    if cache_path:
        cache[key] = best.as_dict()
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best
