"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/bah.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

import paper_2411_15897_gb300 as bah
from paper_2411_15897_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "bah.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bah_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def built():
    try:
        _build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    return _build.build()


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    decl = declared_symbols()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(bah.EXPORTS) == decl


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(bah, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bah, "_lib", None)
    with pytest.raises(RuntimeError):
        bah.lib()


def test_default_options_follow_the_paper(built):
    monkey = bah.bah_default_opts()
    assert monkey.nu_pre == 1 and monkey.nu_post == 2
    assert list(monkey.jacobi_w[:3]) == [0.8, 0.8, 0.3]          # Sec. 4.4.1
    assert monkey.restart == 20 and monkey.precision == bah.BAH_MIXED
    assert bah.status_string(bah.BAH_ERR_ARG) == "BAH_ERR_ARG"


def test_3d_option_checks_run_before_any_device_call(built):
    """3-D contexts need the mixed intergrid of Eq. 4.4 (the paper's 3-D
    transfer), the FP64 Krylov basis and at least two levels; each violation is
    reported by bah_create before it touches a device."""
    import numpy as np
    n = (8, 8, 8)
    med = [np.full(n[::-1], v) for v in (2.0, 1.0, 1.0, 0.0)]
    cases = [(dict(intergrid=bah.BAH_INTERGRID_BILINEAR), bah.BAH_ERR_UNSUPPORTED),
             (dict(intergrid=bah.BAH_INTERGRID_MIXED, krylov_arith=bah.BAH_KRYLOV_DF), bah.BAH_ERR_UNSUPPORTED),
             (dict(intergrid=bah.BAH_INTERGRID_MIXED, levels=1), bah.BAH_ERR_ARG),
             (dict(intergrid=bah.BAH_INTERGRID_MIXED, levels=4), bah.BAH_ERR_ARG)]
    for kw, want in cases:
        with pytest.raises(bah.BahError) as e:
            bah.bah_create(n, (0.1, 0.1, 0.1), *med, 3.0, bah.bah_default_opts(**kw))
        assert e.value.status == want, (kw, bah.last_error())
