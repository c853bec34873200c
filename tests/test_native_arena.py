"""The workspace arena of libvl (vl::Arena in csrc/runtime.cu: a first-fit sub-allocator
over the caller's workspace, which every handle and temporary comes from) under a
randomised alloc/release sequence. tests/native/arena_fuzz.cpp links the built library and
checks, after every operation, that live blocks are aligned, in range and disjoint, that
in_use and peak are exact and that exhaustion is reported only when no hole fits; after
releasing everything the free space must coalesce into one block. Host code only."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_arena_fuzz(tmp_path):
    from paper_2310_12000_gb300 import build
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    lib = build.build()
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build.nvcc())), "include")
    exe = tmp_path / "arena_fuzz"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", build.CSRC, "-I", cuda_inc,
                    os.path.join(HERE, "native", "arena_fuzz.cpp"), lib, f"-Wl,-rpath,{os.path.dirname(lib)}",
                    "-o", str(exe)], check=True)
    for seed in (1, 2, 3):
        r = subprocess.run([str(exe), str(seed)], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
