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


def _desc(mech, **bad):
    """A chem_mech_desc of mech's arrays, with the named arrays replaced."""
    import ctypes
    import numpy as np
    from paper_2312_13513_gb300 import _lib
    fields = {"elem_mass": (mech.elem_mass, np.float64), "comp": (mech.comp, np.int32),
              "nasa_lo": (mech.nasa_lo, np.float64), "nasa_hi": (mech.nasa_hi, np.float64),
              "rtype": (mech.rtype, np.int32), "reac": (mech.reac, np.int32), "prod": (mech.prod, np.int32),
              "A": (mech.A, np.float64), "b": (mech.b, np.float64), "Ea": (mech.Ea, np.float64),
              "troe": (mech.troe, np.float64), "has_t2": (mech.has_t2, np.int32), "eff": (mech.eff, np.float64)}
    keep = {k: np.ascontiguousarray(bad.get(k, v), dtype=t) for k, (v, t) in fields.items()}
    d = _lib.MechDesc(mech.ns, mech.ne, mech.nr, *[keep[k].ctypes.data_as(ctypes.c_void_p) for k in fields])
    return d, keep


def test_mechanism_descriptions_are_validated_on_the_host():
    """chem_load_mechanism_desc checks the description before any device work: each corruption
    below is CHEM_EINVAL with a message naming it; the intact H2 and CH4 descriptions pass the
    checks (on a host without a GPU they then fail at the upload, CHEM_ECUDA)."""
    import ctypes
    import numpy as np
    from paper_2312_13513_gb300 import _lib
    from synth.mechanism import ch4_mechanism, h2_mechanism
    L = _lib.load()
    m = h2_mechanism()
    j3 = int(np.nonzero(m.rtype == 1)[0][0])     # a third-body reaction
    jt = int(np.nonzero(m.rtype == 2)[0][0])     # the fall-off reaction

    def with_(arr, idx, v):
        a = np.array(arr, copy=True)
        a[idx] = v
        return a

    cases = {
        "efficiency": dict(eff=with_(m.eff, (j3, 0), -0.5)),
        "efficiency NaN": dict(eff=with_(m.eff, (j3, 1), np.nan)),
        "Troe NaN": dict(troe=with_(m.troe, (jt, 3), np.nan)),
        "Troe T3": dict(troe=with_(m.troe, (jt, 4), 0.0)),
        "has_t2": dict(has_t2=with_(m.has_t2, jt, 2)),
        "element count": dict(comp=with_(m.comp, (0, 0), -1)),
        "atomic mass": dict(elem_mass=with_(m.elem_mass, 0, np.inf)),
        "species index": dict(reac=with_(m.reac, (0, 0), m.ns)),
        "empty side": dict(prod=with_(m.prod, 0, -1)),
        "Arrhenius": dict(A=with_(m.A, 0, -1.0)),
        "reaction type": dict(rtype=with_(m.rtype, 0, 3)),
        "NASA": dict(nasa_hi=with_(m.nasa_hi, (0, 2), np.inf)),
    }
    h = ctypes.c_void_p()
    for what, bad in cases.items():
        d, _ = _desc(m, **bad)
        rc = L.chem_load_mechanism_desc(ctypes.byref(d), ctypes.byref(h))
        assert rc == _lib.CHEM_EINVAL, what
        assert L.chem_last_error(), what
    for mech in (m, ch4_mechanism()):
        d, _ = _desc(mech)
        rc = L.chem_load_mechanism_desc(ctypes.byref(d), ctypes.byref(h))
        assert rc != _lib.CHEM_EINVAL, L.chem_last_error()
        if rc == _lib.CHEM_OK:
            L.chem_free_mechanism(h)


def test_mesh_descriptions_are_validated_on_the_host():
    """chem_fvmesh_create checks face addressing and patch types before any device work; the
    intact mesh passes the checks (on a host without a GPU it then fails at the upload)."""
    import copy
    import paper_2312_13513_gb300 as cg
    from paper_2312_13513_gb300 import _lib
    from synth.mesh import box_mesh
    m = box_mesh(4, 3, 2, seed=1, permute=True)

    def bad(**kw):
        b = copy.deepcopy(m)
        for k, (i, v) in kw.items():
            getattr(b, k)[i] = v
        return b

    cases = {"owner not below neighbour": bad(owner=(0, int(m.neighbour[0]))),
             "neighbour outside": bad(neighbour=(1, m.n_cells)),
             "owner negative": bad(owner=(2, -1)),
             "boundary cell outside": bad(b_cell=(0, m.n_cells)),
             "patch type": bad(b_type=(3, 2))}
    for what, mesh in cases.items():
        try:
            cg.FvMesh(mesh)
        except cg.ChemError as e:
            assert e.code == _lib.CHEM_EINVAL, what
        else:
            raise AssertionError(f"{what}: accepted")
    try:
        cg.FvMesh(m).close()
    except cg.ChemError as e:
        assert e.code != _lib.CHEM_EINVAL, str(e)


def test_a_missing_library_fails_loudly(monkeypatch, tmp_path):
    """With the CUDA library unavailable, the API raises instead of falling back to anything:
    there is no CPU path behind the binding."""
    import pytest
    import paper_2312_13513_gb300 as cg
    from paper_2312_13513_gb300 import _lib
    from synth.mechanism import h2_mechanism
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib._build, "build", lambda *a, **k: str(tmp_path / "libchem.so"))
    with pytest.raises(ImportError):
        _lib.load()
    with pytest.raises(ImportError):
        cg.Mechanism(h2_mechanism())
