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


def test_argument_validation_without_gpu():
    """Invalid arguments are rejected with QS_EINVAL before any CUDA call."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("_qs_build", os.path.join(ROOT, "paper_2108_11989_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    lib = ctypes.CDLL(b.build())

    class Geom(ctypes.Structure):
        _fields_ = [("L", ctypes.c_int), ("T", ctypes.c_int), ("cstar_mask", ctypes.c_int),
                    ("t_antiperiodic", ctypes.c_int), ("device", ctypes.c_int)]

    h = ctypes.c_void_p()
    for L, T, mask in [(3, 4, 7), (4, 1, 7), (4, 4, 6), (4, 4, 9), (512, 512, 7)]:
        assert lib.qs_create_lattice(ctypes.byref(Geom(L, T, mask, 0, 0)), None, ctypes.byref(h)) == -1
    assert lib.qs_create_lattice(None, None, ctypes.byref(h)) == -1
    assert lib.qs_apply_Q_batch(None, 1, 0, None) == -1
    lib.qs_lowmodes_at_mass.argtypes = [ctypes.c_void_p, ctypes.c_double] + [ctypes.c_void_p] * 5
    assert lib.qs_lowmodes_at_mass(None, 0.0, None, None, None, None, None) == -1
    lib.qs_pfaffian_sign.argtypes = [ctypes.c_void_p, ctypes.c_double] + [ctypes.c_void_p] * 3
    assert lib.qs_pfaffian_sign(None, 0.0, None, None, None) == -1
    assert lib.qs_mlp_create(0, 8, 4, 16, None, ctypes.byref(h)) == -1
    assert lib.qs_mlp_create(8, 8, 1, 16, None, ctypes.byref(h)) == -1
    lib.qs_apply_Q_norm2_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_double] + [ctypes.c_void_p] * 2 + \
        [ctypes.c_int] * 2 + [ctypes.c_void_p]
    assert lib.qs_apply_Q_norm2_noalloc(None, 0.0, None, None, 1, 0, None) == -1
    assert lib.qs_destroy_lattice(None) == 0
    lib.qs_n_sites.restype = ctypes.c_int64
    assert lib.qs_n_sites(None) == 0
