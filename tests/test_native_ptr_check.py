"""The pointer-placement rule of the library on the host: device memory is used in place
only on the context's own device (another GPU's memory is refused, never read across), managed
memory on any device, host and unregistered memory never. No GPU."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
# cudaMemoryType values of the CUDA runtime
UNREGISTERED, HOST, DEVICE, MANAGED = 0, 1, 2, 3


def test_device_memory_only_on_the_context_device(tmp_path):
    from paper_2310_12000_gb300 import build
    exe = tmp_path / "ptr_check_host"
    r = subprocess.run([build.nvcc(), *build.ARCH, "-std=c++17", "-I", build.CSRC,
                        os.path.join(HERE, "native", "ptr_check_host.cu"), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stdout + r.stderr)
    cases = [(DEVICE, 0, 0, 1), (DEVICE, 1, 0, 0), (DEVICE, 0, 3, 0), (DEVICE, 5, 5, 1),
             (MANAGED, 2, 0, 1), (MANAGED, -2, 1, 1), (HOST, 0, 0, 0), (UNREGISTERED, 0, 0, 0)]
    inp = "\n".join(f"{a} {b} {c}" for a, b, c, _ in cases) + "\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=60,
                         check=True).stdout.split()
    assert [int(v) for v in out] == [e for *_, e in cases]
