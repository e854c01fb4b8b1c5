"""The C-ABI library builds, loads and exports every function include/cusci.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_2604_15768_gb300 import build as B
from paper_2604_15768_gb300 import cusci

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "cusci.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cusci_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    names = declared_functions()
    assert names == cusci.exported_names()


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert lib.cusci_version
