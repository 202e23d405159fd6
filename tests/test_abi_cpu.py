"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point include/life.h declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "life.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(life_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_1905_06234_gb300 import _native
    assert sorted(declared_symbols()) == sorted(_native.EXPORTS)


def test_library_exports_every_declared_symbol():
    from paper_1905_06234_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    lib.life_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.life_version()


def test_no_oracle_in_product_path():
    # The product package must not import or link the oracle.
    pkg = os.path.join(ROOT, "paper_1905_06234_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f
