"""The C-ABI library builds, loads and exports every entry point that
include/sphgb.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sphgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_1404_2303_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # every declared function has a Python signature (the binding mirrors the ABI)
    assert set(names) <= set(_lib.SIGNATURES)


def test_default_params_and_status_strings():
    from paper_1404_2303_gb300 import _lib, default_params
    lib = _lib.load()
    p = default_params()
    assert p.n_ngb == 48.0 and abs(p.gamma - 5 / 3) < 1e-7
    assert p.split_count == 300 and abs(p.split_frac - 0.875) < 1e-7
    for code in range(-8, 1):
        assert lib.sph_status_string(code)
