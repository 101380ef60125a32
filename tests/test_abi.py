"""The C-ABI library builds, loads without a GPU, and exports every symbol the header declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(lsg_[A-Za-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2004_13961_gb300 import lsg
    L = lsg.load()
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    assert set(lsg.SYMBOLS) == declared


def test_host_only_calls_without_gpu():
    from paper_2004_13961_gb300 import lsg
    L = lsg.load()
    assert L.lsg_version() >= 100
    assert L.lsg_status_string(-4).decode().startswith("ILU(0) breakdown")
    # footprint model: pure host arithmetic
    fp2 = lsg.footprint_bytes(2, 512, 8)
    fp3 = lsg.footprint_bytes(3, 128, 6, precision=lsg.MIXED_TF32)
    assert 0.9e9 < fp2 < 4e9
    assert 30e9 < fp3 < 120e9
    assert lsg.footprint_bytes(4, 10, 2) == 0  # invalid dimension


def test_oracle_and_library_share_no_code():
    """The oracle never includes or links the CUDA sources and vice versa."""
    osrc = open(os.path.join(ROOT, "oracle", "lsg_oracle.c")).read()
    assert "lsg.h" not in osrc and "csrc" not in osrc
    for fn in os.listdir(os.path.join(ROOT, "paper_2004_13961_gb300", "csrc")):
        txt = open(os.path.join(ROOT, "paper_2004_13961_gb300", "csrc", fn)).read()
        assert "oracle" not in txt.lower(), fn
    for fn in ("lsg.py", "build.py", "workloads.py", "__init__.py"):
        txt = open(os.path.join(ROOT, "paper_2004_13961_gb300", fn)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, fn
