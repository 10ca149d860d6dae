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
