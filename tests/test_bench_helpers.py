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
