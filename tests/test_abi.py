"""The C ABI library loads without a GPU and exports every entry point the header
declares; the Python binding wraps exactly those names (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "splx.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(splx_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_2606_18588_gb300 import splx as S
    lib = ctypes.CDLL(S.LIB_PATH)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(S.EXPORTED) == names


def test_status_strings_without_gpu():
    from paper_2606_18588_gb300 import splx as S
    assert S._lib.splx_strerror(S.ERR_CAPACITY) == b"pair capacity exceeded"
    assert S._lib.splx_strerror(12345) == b"unknown status"
