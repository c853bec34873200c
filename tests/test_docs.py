"""The design document names kernels and files that exist: every `*_kernel` it mentions is
defined in csrc/, and every file name it puts in backticks is present in the repository."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_design_document_references_resolve():
    doc = open(os.path.join(ROOT, "DESIGN.md")).read()
    src = "".join(open(f).read() for f in glob.glob(os.path.join(ROOT, "paper_2310_12000_gb300", "csrc", "*")))
    kernels = set(re.findall(r"`([a-z_0-9]+_kernel)\b", doc))
    assert kernels and not [k for k in kernels if k not in src]
    files = set(re.findall(r"`([A-Za-z_0-9/]+\.(?:cu|cuh|h|py|md|json|cpp))`", doc))
    missing = [f for f in files
               if not [p for p in glob.glob(os.path.join(ROOT, "**", os.path.basename(f)), recursive=True)
                       if "_work" not in p]]
    assert files and not missing, missing
