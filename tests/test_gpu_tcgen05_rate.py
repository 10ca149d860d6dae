"""Tensor-core rate at the shapes of a block Gram-Schmidt step.

Builds tests/tcgen05_rate.cu with nvcc for sm_103a and runs it: an exact
check of one bfloat16 tcgen05.mma product read back from tensor memory
(N = 32 and N = 256), then the rate of M = 128, K = 16 instructions at
N = 16 ... 256 with one CTA per SM.  The rates are printed (pytest -s); the
test asserts the exact check, that every wait completed, and that wider N
never lowers the rate by more than the timing noise.  The numbers feed the
cost model of an FP64-accurate (split-operand) block Gram-Schmidt on the
tensor cores.
"""
import json
import os
import shutil
import subprocess

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


def test_tcgen05_mma_exact_and_rate(tmp_path):
    exe = str(tmp_path / "tcgen05_rate")
    subprocess.run([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-o", exe,
                    os.path.join(HERE, "tcgen05_rate.cu")], check=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    lines = [json.loads(s) for s in out.stdout.splitlines() if s.startswith("{")]
    print("\n".join(json.dumps(x) for x in lines))
    assert out.returncode == 0, out.stdout + out.stderr
    checks = [x for x in lines if x.get("check")]
    assert [c["n"] for c in checks] == [32, 256]
    assert all(c["maxerr"] == 0 and c["timeout"] == 0 for c in checks)
    rates = {x["n"]: x["tflops"] for x in lines if not x.get("check")}
    assert sorted(rates) == [16, 32, 64, 128, 256]
    assert all(r > 0 for r in rates.values())
    assert rates[256] >= 0.9 * rates[16]
