"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(efe_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2607_06848_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert "efe_setup" in declared and "efe_chfsi" in declared and len(declared) >= 12
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2607_06848_gb300 import efe
    declared = _declared()
    assert declared <= set(efe.SIGNATURES), sorted(declared - set(efe.SIGNATURES))


def test_setup_rejects_bad_arguments_without_launching():
    # argument errors are detected before any device work, so this runs on CPU
    from paper_2607_06848_gb300 import efe
    lib = efe.load()
    mesh = efe.efe_mesh(2.0, (ctypes.c_int * 3)(4, 4, 4), 0, 0)     # degree 0 is invalid
    xyz = (ctypes.c_double * 3)(4.0, 4.0, 4.0)
    z = (ctypes.c_double * 1)(4.0)
    at = efe.efe_atoms(1, xyz, z)
    ctx = ctypes.c_void_p()
    st = lib.efe_setup(ctypes.byref(mesh), ctypes.byref(at), None, None, None, ctypes.byref(ctx))
    assert st == 1 and not ctx.value
    assert b"degree" in lib.efe_last_error(None)
    mesh.degree = 4
    en = efe.efe_enrichment(1, 1.2, 5.0, 0.33)                        # support leaves an 8-bohr box
    st = lib.efe_setup(ctypes.byref(mesh), ctypes.byref(at), ctypes.byref(en), None, None, ctypes.byref(ctx))
    assert st == 1 and b"leaves the box" in lib.efe_last_error(None)
