"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/holstein.h (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^(?!typedef|#)[\w \t*]+?\b(\w+)\s*\(", src, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hol_create", "hol_destroy", "hol_set_field", "fermion_matvec",
                     "cg_solve", "force"):
        assert required in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2203_01291_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_2203_01291_gb300 import _abi
    assert set(_abi.SIGNATURES) == set(declared_functions())


def test_no_oracle_import_in_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2203_01291_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_context_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2203_01291_gb300 as hg
    with pytest.raises(RuntimeError):
        hg.Context(L=4, Ltau=8)
