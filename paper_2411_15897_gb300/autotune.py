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

``tune_cycle`` chooses the multigrid cycle, its sweep counts, the shift alpha
(Eq. 2.8) and the FGMRES restart length.  These change the iteration count,
not only the cost of an iteration, so each candidate is timed on complete
solves to the tolerance (of a sample of the workload's sources), as the paper
chooses its shift by a search at a resolution of 0.1 (Sec. 4.4.3).
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


# ---------------------------------------------------------------------------
# cycle, shift and restart: timed on complete solves
# ---------------------------------------------------------------------------
@dataclass
class CycleChoice:
    settings: dict                    # solver options (cycle, nu_pre, nu_post, shift_alpha, restart)
    seconds: float                    # per source, to the tolerance
    iters: int
    table: list = field(default_factory=list)   # (settings, seconds, iters) of every candidate

    def as_dict(self):
        return {"settings": self.settings, "seconds": self.seconds, "iters": self.iters, "table": self.table}


def cycle_candidates(alphas=(0.6, 0.7, 0.8, 0.9, 1.0), cycles=(("V", 1, 2), ("V", 1, 3), ("W", 1, 2)),
                     restarts=(10, 20)):
    """The search grid: every cycle (type, nu_pre, nu_post) x shift x restart."""
    out = []
    for cyc, n1, n2 in cycles:
        for a in alphas:
            for m in restarts:
                out.append({"cycle": 1 if cyc == "W" else 0, "nu_pre": n1, "nu_post": n2,
                            "shift_alpha": float(a), "restart": int(m)})
    return out


def time_solve(problem, settings, opts, sources, rtol=1e-6, maxit=20000):
    """(seconds per source, max iterations) of one solve of ``sources`` (indices
    into problem.sources, one batch) to ``rtol`` with the given settings, on
    the current CUDA device (one untimed solve first); inf if it does not
    converge."""
    import numpy as np
    import torch

    import workloads as W
    from . import BAH_OK, Solver, bah_solve

    nb = len(sources)
    s = Solver.from_problem(problem, **dict(opts, **settings, rhs_block=nb, maxit=maxit))
    b = torch.from_numpy(np.stack([W.point_source(problem, problem.sources[q]) for q in sources])).cuda()
    x = torch.zeros_like(b)
    st, stats = bah_solve(s.ctx, b, x, nb, rtol)
    if st != BAH_OK:
        s.close()
        return float("inf"), max(q["iters"] for q in stats)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    st, stats = bah_solve(s.ctx, b, x, nb, rtol)
    e1.record(stream)
    e1.synchronize()
    s.close()
    return e0.elapsed_time(e1) * 1e-3 / nb, max(q["iters"] for q in stats)


def tune_cycle(problem, opts=None, candidates=None, sample=4, measure=time_solve) -> CycleChoice:
    """Fastest settings per source to the tolerance over ``candidates``
    (default: cycle_candidates()), timed on up to ``sample`` of the problem's
    sources spread over its source list, solved as one batch."""
    opts = {k: v for k, v in dict(opts or {}).items()
            if k not in ("cycle", "nu_pre", "nu_post", "shift_alpha", "restart", "rhs_block", "maxit")}
    nsrc = max(1, len(problem.sources))
    k = min(sample, nsrc)
    sources = sorted({int(round(i * (nsrc - 1) / max(k - 1, 1))) for i in range(k)})
    table, best = [], None
    for cand in (candidates or cycle_candidates()):
        sec, its = measure(problem, cand, opts, sources)
        table.append((cand, sec, its))
        if best is None or sec < best.seconds:
            best = CycleChoice(dict(cand), sec, its)
    best.table = table
    return best
