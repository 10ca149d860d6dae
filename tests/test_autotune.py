"""The batched-solve autotuner's search and cache (no GPU: the timing
function is replaced by a cost model)."""
import pytest

import workloads as W
from paper_2411_15897_gb300 import autotune


def test_candidates_cover_powers_of_two_and_the_source_count():
    assert autotune.candidates(64) == [1, 2, 4, 8, 16, 32, 64]
    assert autotune.candidates(12) == [1, 2, 4, 8, 12]
    assert autotune.candidates(1) == [1]
    assert autotune.candidates(1000) == [1, 2, 4, 8, 16, 32, 64, 128, 256]


def test_tune_picks_the_cheapest_and_caches_it(tmp_path):
    p = W.layered(64, 32, 4, seed=23, abc=6, nsrc=12, src_spacing=4)
    calls = []

    def model(problem, rb, env, opts, iters):
        calls.append((rb, tuple(sorted(env.items()))))
        # launches amortised over the batch, plus a per-source cost growing with the batch;
        # staging off costs 5 %
        return (1.0 / rb + 0.02 * rb) * (1.05 if env.get("BAH_STAGED") == "0" else 1.0)

    cache = tmp_path / "tune.json"
    c = autotune.tune(p, opts={"precision": 1}, iters=5, measure=model, cache_path=str(cache), device="test")
    assert (c.rhs_block, c.variant) == (8, "default")
    assert len(c.table) == len(autotune.candidates(12)) * len(autotune.VARIANTS) == len(calls)
    assert all(rb <= 12 for rb, _ in calls)

    def fail(*a):
        raise AssertionError("the cached choice must be used")
    c2 = autotune.tune(p, opts={"precision": 1}, iters=5, measure=fail, cache_path=str(cache), device="test")
    assert (c2.rhs_block, c2.variant, c2.cost) == (c.rhs_block, c.variant, c.cost)
    # another precision is another key
    with pytest.raises(AssertionError):
        autotune.tune(p, opts={"precision": 0}, iters=5, measure=fail, cache_path=str(cache), device="test")


def test_tune_cycle_times_complete_solves_and_keeps_the_fastest():
    """The cycle/shift/restart search times each candidate on a sample of the
    sources spread over the source list and keeps the fastest per source; a
    candidate that does not converge (infinite time) is never chosen."""
    p = W.layered(64, 32, 4, seed=23, abc=6, nsrc=12, src_spacing=4)
    seen = []

    def model(problem, cand, opts, sources):
        seen.append((tuple(sorted(cand.items())), tuple(sources)))
        assert "rhs_block" not in opts and "shift_alpha" not in opts
        if cand["cycle"] == 1 and cand["shift_alpha"] < 0.7:
            return float("inf"), 20000
        its = 1000 * (1 + abs(cand["shift_alpha"] - 0.8)) / (2 if cand["cycle"] == 1 else 1)
        per_iter = (1.0 + 0.02 * cand["restart"]) * (2.3 if cand["cycle"] == 1 else 1.0 + 0.2 * (cand["nu_post"] - 2))
        return its * per_iter * 1e-6, int(its)

    c = autotune.tune_cycle(p, opts={"precision": 1, "shift_alpha": 0.3, "rhs_block": 8}, sample=4, measure=model)
    assert len(seen) == len(autotune.cycle_candidates())
    assert all(src == (0, 4, 7, 11) for _, src in seen)
    assert c.settings["shift_alpha"] == 0.8 and c.settings["restart"] == 10
    assert c.seconds == min(s for _, s, _ in c.table)
