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


def _struct_fields(name):
    """(field, C type, array length) of `typedef struct name {...} name;` in
    the header, comments removed."""
    src = open(os.path.join(ROOT, "include", "sphgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    body = re.search(r"typedef struct " + name + r"\s*\{(.*?)\}\s*" + name + ";", src, re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(int32_t|int64_t|float|double)\s+(\w+)(?:\[(\d+)\])?$", decl)
        assert m, decl
        out.append((m.group(2), m.group(1), int(m.group(3)) if m.group(3) else 0))
    return out


def test_ctypes_structs_mirror_the_header():
    """The binding's SphParams / SphStats have the header's fields, in order,
    with the same types: the structs cross the C ABI by pointer."""
    import ctypes as C
    from paper_1404_2303_gb300 import _lib
    ctype = {"int32_t": C.c_int32, "int64_t": C.c_int64, "float": C.c_float, "double": C.c_double}
    for cname, py in (("sph_params", _lib.SphParams), ("sph_stats", _lib.SphStats)):
        want = _struct_fields(cname)
        got = py._fields_
        assert [f for f, _, _ in want] == [f for f, _ in got], cname
        for (f, t, k), (_, pt) in zip(want, got):
            assert pt == (ctype[t] * k if k else ctype[t]), (cname, f)


def test_default_params_of_the_optimised_paths():
    from paper_1404_2303_gb300 import default_params
    p = default_params()
    assert p.use_graph == 1 and p.kahan == 1 and p.sorted_sweep == 1
    assert p.pair_list_cap == 256 and p.list_cap == 4096 and p.sweep_lists == 0x08
    assert p.sweep_cap == 128 and p.warps_per_cta == 8 and p.block_max == 64
