"""Host-side helpers of bench.py (no GPU)."""
import numpy as np
import pytest

import workloads as W


def test_rhs_count_from_vector_length():
    """The number of right-hand sides comes from the buffer's size, not its
    rank: one 3-D vector (4, n3, n2, n1) is one right-hand side, a stack of 2-D
    vectors (k, 3, n2, n1) is k."""
    import bench
    n3 = (6, 5, 4)
    v3 = np.zeros(W.padded_shape(n3), dtype=np.complex128)
    assert v3.ndim == 4 and bench.rhs_count(v3, v3.size) == 1
    n2 = (6, 5)
    v2 = np.zeros((7,) + W.padded_shape(n2), dtype=np.complex128)
    assert v2.ndim == 4 and bench.rhs_count(v2, v2[0].size) == 7
    torch = pytest.importorskip("torch")
    assert bench.rhs_count(torch.zeros(3 * v3.size), v3.size) == 3
    with pytest.raises(ValueError):
        bench.rhs_count(np.zeros(v3.size + 1), v3.size)


def test_presets_keep_the_2d_benchmark_and_give_c5_the_3d_cycle(monkeypatch):
    """The default line keeps the 2-D benchmark's tuned cycle with the FP64
    Krylov basis; --config c4 takes the library's own cycle (V(1,2), shift by
    level count); --config c5 gets the paper's 3-D multigrid (W(2,2), mixed
    intergrid, Jacobi 0.8/0.8/0.2) on 5 levels; explicit flags override a
    preset."""
    import bench
    fields = ("levels", "alpha", "cycle", "nu", "jacobi", "intergrid", "krylov", "restart")
    monkeypatch.setattr("sys.argv", ["bench.py"])
    a = bench.parse()
    assert tuple(getattr(a, f) for f in fields) == (0, 0.8, "V", "1,3", "0.8,0.8,0.3", "bilinear", "fp64", 10)
    monkeypatch.setattr("sys.argv", ["bench.py", "--config", "c4"])
    a = bench.parse()
    assert tuple(getattr(a, f) for f in fields) == (0, -1.0, "V", "1,2", "0.8,0.8,0.3", "bilinear", "fp64", 20)
    monkeypatch.setattr("sys.argv", ["bench.py", "--config", "c5"])
    a = bench.parse()
    assert tuple(getattr(a, f) for f in fields) == (5, 0.4, "W", "2,2", "0.8,0.8,0.2", "mixed", "fp64", 20)
    monkeypatch.setattr("sys.argv", ["bench.py", "--config", "c5", "--alpha", "0.3", "--nu", "1,2"])
    a = bench.parse()
    assert (a.alpha, a.nu, a.cycle) == (0.3, "1,2", "W")
