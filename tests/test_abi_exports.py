"""The C-ABI library loads and exports every function include/bfhe.h declares
(no GPU needed: nothing is called but the loader)."""

import ctypes
import os
import re

from paper_2204_12201_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bfhe.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bfhe_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = build.lib_path()
    if not os.path.exists(path):
        build.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    from paper_2204_12201_gb300 import bfhe
    src = open(bfhe.__file__).read()
    missing = [n for n in declared() if '"%s"' % n not in src]
    assert not missing, missing
