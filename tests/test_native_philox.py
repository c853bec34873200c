"""The CUDA side's Philox4x64-10 (csrc/vl_device.cuh), run on the host, against numpy's Philox
bit generator (the published Philox4x64-10, Salmon et al. 2011). The probe and simulation
kernels draw every random number from this function, so with the oracle's own generator
pinned to numpy as well, both sides are tied to the same published definition. No GPU."""
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
M64 = (1 << 64) - 1


def _numpy_block(ctr, key):
    """The block numpy produces for counter `ctr` (numpy increments before each block)."""
    c = list(ctr)
    c[0] -= 1
    for w in range(3):                      # undo the increment with borrow
        if c[w] >= 0:
            break
        c[w] += 1 << 64
        c[w + 1] -= 1
    c = [x & M64 for x in c]
    bg = np.random.Philox(counter=np.array(c, np.uint64), key=np.array(key, np.uint64))
    return [int(v) for v in bg.random_raw(4)]


def test_cuda_philox_matches_numpy(tmp_path):
    from paper_2310_12000_gb300 import build
    exe = tmp_path / "philox_host"
    r = subprocess.run([build.nvcc(), *build.ARCH, "-std=c++17", "-I", build.CSRC,
                        os.path.join(HERE, "native", "philox_host.cu"), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stdout + r.stderr)
    rng = np.random.default_rng(0)
    cases = [((0, 0, 0, 0), (0, 0)), ((1, 0, 0, 0), (1, 0)), ((5, 0, 0, 0), (7, 9)),
             ((2**64 - 1, 3, 2**63, 1), (2**64 - 1, 12345)), ((12, 3, 1, 0), (1, 0))]
    cases += [(tuple(int(x) for x in rng.integers(0, 2**63, 4, dtype=np.int64)),
               tuple(int(x) for x in rng.integers(0, 2**63, 2, dtype=np.int64))) for _ in range(40)]
    inp = "".join(" ".join(str(v) for v in (*c, *k)) + "\n" for c, k in cases)
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=60, check=True).stdout
    got = [[int(v) for v in line.split()] for line in out.strip().splitlines()]
    assert len(got) == len(cases)
    for (c, k), g in zip(cases, got):
        assert g == _numpy_block(c, k), (c, k)
