"""The C-ABI library builds, loads and exports every entry point include/lks.h declares (no GPU).

Only non-compute calls are made here (status strings); everything that touches the device is in
the gpu-marked tests.
"""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lks.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^LKS_API\s+[\w\s\*]+?\b(lks_\w+)\s*\(", src, flags=re.M)))


def _have_nvcc():
    import shutil
    return shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")


@pytest.mark.skipif(not _have_nvcc(), reason="nvcc not available")
def test_library_exports_every_declared_symbol():
    from paper_2601_18272_gb300 import lks
    L = lks.load()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    lib = ctypes.CDLL(lks.library_path())
    for n in names:
        getattr(lib, n)


@pytest.mark.skipif(not _have_nvcc(), reason="nvcc not available")
def test_status_strings():
    from paper_2601_18272_gb300 import lks
    assert lks.lks_status_string(0) == "ok"
    assert "unsupported" in lks.lks_status_string(9)
    assert lks.lks_status_string(1234) == "unknown status"


def test_problem_struct_mirrors_header():
    """Field order and types of the ctypes mirror follow the C struct in include/lks.h."""
    from paper_2601_18272_gb300.lks import lks_problem
    src = open(HEADER).read()
    body = src[src.index("typedef struct lks_problem {"):src.index("} lks_problem;")]
    names = []
    for line in body.splitlines()[1:]:
        line = line.split("/*")[0].strip().rstrip(";")
        if not line:
            continue
        decl = line.split(None, 1)
        if decl[0] == "unsigned" or decl[0] == "size_t" or decl[0] in ("int", "double"):
            for part in decl[1].split(","):
                names.append(part.strip().split("[")[0].strip())
    assert [f[0] for f in lks_problem._fields_] == names
