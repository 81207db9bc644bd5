"""The C-ABI library loads on any host and exports every function include/chem.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(chem_[a-z0-9_]+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2312_13513_gb300 import _lib
    L = _lib.load()
    names = declared_functions()
    assert len(names) >= 8
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(_lib.SIGNATURES) <= set(names)


def test_last_error_is_callable_without_gpu():
    from paper_2312_13513_gb300 import _lib
    L = _lib.load()
    assert isinstance(L.chem_last_error(), (bytes, type(None)))
    # argument validation happens before any device work
    rc = L.chem_mechanism_info(None, None, None, None)
    assert rc == _lib.CHEM_EINVAL
    assert b"NULL" in L.chem_last_error()
