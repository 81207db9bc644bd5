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


def test_every_entry_point_rejects_null_arguments_before_device_work():
    """The header's error contract on a host without a GPU: called with NULL handles and pointers
    (sizes 1, scalars 1.0), every entry point returns CHEM_EINVAL and leaves a message, without
    touching the device.  The two calls that take no handle (the FMA-peak probe, the error
    query) are left out."""
    import ctypes
    from paper_2312_13513_gb300 import _lib
    L = _lib.load()
    checked = 0
    for name, (_, argtypes) in _lib.SIGNATURES.items():
        if name in ("chem_fp64_fma_peak", "chem_last_error"):
            continue
        args = []
        for a in argtypes:
            if a in (ctypes.c_double, ctypes.c_float):
                args.append(1.0)
            elif a in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(a, ctypes._Pointer):
                args.append(None)
            else:
                args.append(1)
        rc = getattr(L, name)(*args)
        assert rc == _lib.CHEM_EINVAL, (name, rc)
        assert L.chem_last_error(), name
        checked += 1
    assert checked >= 45
