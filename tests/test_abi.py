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
    assert o.cg_tol == 1e-6 and o.newton_tol == 1e-9 and o.nugget == -1.0 and o.lik_shape == 1.0
    assert o.newton_eta_max == 0.1


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


def test_binding_structs_and_constants_match_the_c_header(tmp_path):
    """The ctypes mirrors of vl_opts and vl_stats have the size and field offsets that a C
    compiler gives the declarations in include/vl.h (a mismatch would corrupt every call), and
    the binding's enum constants have the header's values."""
    import shutil
    import subprocess

    import paper_2310_12000_gb300 as vl
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"vl_opts": vl.Opts, "vl_stats": vl.Stats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "vl.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    consts = ["COV_EXPONENTIAL", "COV_MATERN15", "LIK_BERNOULLI_LOGIT", "LIK_POISSON_LOG", "LIK_GAMMA_LOG", "PREC_VADU",
              "PREC_LVA", "PREC_LRAC", "FP64", "FP32_REFINE", "OP_A", "OP_PINV", "OP_B", "OP_BT", "OP_BINV",
              "OP_BTINV", "OP_SIGMA", "OP_A2", "SOLVE_AUTO", "SOLVE_SHARED", "SOLVE_CLUSTER", "SOLVE_GRID",
              "SOLVE_GRID_ALL", "SOLVE_TILE"]
    for name in consts:
        lines.append(f'  printf("const {name} %d\\n", (int)VL_{name});')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name in consts:
        assert got[("const", name)] == getattr(vl, name), name
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libvl.so there is no fallback: loading the library and making a context raise."""
    from paper_2310_12000_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "lib_path", lambda: str(tmp_path / "libvl.so"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        _lib.library()
    with pytest.raises(ImportError):
        _lib.Context(0, ws_bytes=1 << 24)
