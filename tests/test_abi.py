"""The C ABI library loads and exports every function include/*.h declares
(no GPU needed: nothing is launched)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fn_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("fn_time_edges", "fn_knn_tree", "fn_rnea_dump", "fn_status_str"):
        assert must in names


def test_library_exports_declared_symbols():
    from paper_2609_22608_gb300 import _build
    _build.build()
    lib = ctypes.CDLL(_build.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.fn_status_str.restype = ctypes.c_char_p
    assert lib.fn_status_str(-1).startswith(b"FN_EINVAL")


def test_oracle_builds_and_is_separate():
    import oracle
    oracle.build()
    # the oracle and the CUDA path share no sources
    csrc = os.path.join(ROOT, "paper_2609_22608_gb300", "csrc")
    for f in glob.glob(os.path.join(csrc, "*")):
        assert "fn_oracle" not in open(f).read()
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        text = open(f).read()
        assert "fn_api.h" not in text and "csrc" not in text
