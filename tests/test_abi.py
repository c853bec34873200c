"""The C-ABI library builds, loads and exports every entry point include/vl.h declares.

No compute call is made here (these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "vl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vl_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_12000_gb300 import build
    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s


def test_version_and_defaults(lib):
    import paper_2310_12000_gb300 as vl
    L = vl.library()
    assert L.vl_version().startswith(b"vl ")
    o = vl.Opts.make()
    assert (o.t, o.s, o.precond, o.precision, o.cg_max_iter) == (50, 100, vl.PREC_VADU, vl.FP64, 1000)
    assert o.cg_tol == 1e-6 and o.newton_tol == 1e-9 and o.nugget == -1.0


def test_context_creation_fails_cleanly_without_gpu(lib):
    from conftest import cuda_available
    if cuda_available():
        pytest.skip("a GPU is present")
    import paper_2310_12000_gb300 as vl
    h = ctypes.c_void_p()
    s = vl.library().vl_ctx_create(0, None, None, 1 << 24, ctypes.byref(h))
    assert s in (2, 6) and not h.value


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    import paper_2310_12000_gb300 as vl
    L = vl.library()
    assert L.vl_ctx_create(0, None, None, 10, None) == 1     # out == NULL / ws too small
    assert L.vl_build_factor(None, None, 10, None, 0, 1.0, 1.0, 5, None, None) == 1
    assert L.vl_find_mode(None, 0, None, None, None, None, None) == 1
