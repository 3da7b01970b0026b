"""The C-ABI library loads and exports every entry point that include/*.h declares
(CPU only: nothing here launches GPU work)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"QS_API\s+[\w\s\*]+?\b(qs_\w+)\s*\(", txt))
    return names


def test_library_exports_all_declared_symbols():
    import importlib.util
    spec = importlib.util.spec_from_file_location("_qs_build", os.path.join(ROOT, "paper_2108_11989_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_symbols()
    assert len(names) >= 8
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    lib.qs_strerror.restype = ctypes.c_char_p
    assert lib.qs_strerror(-7).decode().startswith("|lambda|")
