"""The C ABI library loads and exports every symbol include/gbx.h declares;
host-only entry points (descriptor, error text) behave. CPU only: nothing
here launches device work."""
import ctypes
import os
import re

import pytest

import paper_1908_01407_gb300 as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(gb.LIB_PATH):
        gb.build_library()
    return gb.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gbx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gb_info|const char \*)\s*(gb_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) > 50
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    names = set(declared_functions()) - {"gb_version"}
    assert names <= set(gb._SIGS), sorted(names - set(gb._SIGS))


def test_descriptor_host_logic(L):
    d = gb.Descriptor()
    assert d.get(gb.F_MASK) == gb.DEFAULT
    d.toggle(gb.F_MASK)
    assert d.get(gb.F_MASK) == gb.SCMP
    d.set(gb.F_MASK, gb.SCMP | gb.STRUCTURE)
    d.toggle(gb.F_MASK)
    assert d.get(gb.F_MASK) == gb.STRUCTURE
    d.toggle(gb.F_INP1)
    assert d.get(gb.F_INP1) == gb.TRAN
    d.toggle(gb.F_OUTP)
    assert d.get(gb.F_OUTP) == gb.REPLACE
    d.set(gb.F_DIRECTION, gb.PULL).set(gb.F_SWITCH_BETA, 14)
    assert d.get(gb.F_DIRECTION) == gb.PULL and d.get(gb.F_SWITCH_BETA) == 14
    with pytest.raises(gb.GBError) as e:
        d.set(gb.F_DIRECTION, 7)
    assert e.value.code == gb.INVALID_VALUE
    with pytest.raises(gb.GBError) as e:
        d.toggle(gb.F_SWITCH_BETA)
    assert e.value.code == gb.INVALID_VALUE
    d.free()


def test_null_arguments_return_codes_not_crashes(L):
    assert L.gb_matrix_nrows(None, None) == gb.NULL_POINTER
    assert L.gb_bfs(None, None, 0, None, None, 0, None, None) == gb.NULL_POINTER
    assert "NULL" in gb.last_error()
    assert L.gb_desc_new(None) == gb.NULL_POINTER
    assert gb.version().startswith("gbx")


def test_teps_metric_matches_paper_table9():
    from tests.conftest import read_golden
    f = read_golden("table12_bfs_teps.txt")
    got = gb.teps(float(f["edges"]), float(f["runtime_ms"]) / 1e3) / 1e6
    want = float(f["mteps"])
    assert abs(got - want) / want < float(f["rel_tol"])
    got_t = gb.teps(float(f["edges"]), float(f["titan_runtime_ms"]) / 1e3) / 1e9
    assert abs(got_t - float(f["titan_gteps"])) / float(f["titan_gteps"]) < 0.005


def test_every_entry_point_rejects_null_handles(L):
    """Each call of the ABI, given NULL for every pointer and 0 for every
    number, returns an error code (NULL_POINTER, or INVALID_VALUE where a
    count of 0 is checked first) without touching a device or crashing."""
    import ctypes as C
    codes = {}
    for name, argtypes in sorted(gb._SIGS.items()):
        f = getattr(L, name)
        args = [None if t in (C.c_void_p, C.c_char_p) or isinstance(t, type(C.POINTER(C.c_int)))
                else t(0) for t in argtypes]
        codes[name] = f(*args)
    bad = {n: c for n, c in codes.items() if c not in (gb.NULL_POINTER, gb.INVALID_VALUE)}
    assert not bad, bad
    assert codes["gb_bfs_multi"] == gb.INVALID_VALUE          # k == 0 is checked before the handles
    assert codes["gb_bfs_batch"] == gb.NULL_POINTER


def test_noalloc_limit_of_the_library_is_the_headers(L):
    """The scratch limit compiled into the library (its size check runs on
    the host, before any device call) equals the GB_NOALLOC_MAX_VERTICES of
    include/gbx.h, which the binding reads."""
    src = open(os.path.join(ROOT, "include", "gbx.h")).read()
    limit = int(re.search(r"#define\s+GB_NOALLOC_MAX_VERTICES\s+(\d+)u?", src).group(1))
    assert gb.NOALLOC_MAX_VERTICES == limit
    p = ctypes.c_void_p(4096)          # never dereferenced: the size check comes first
    rc = L.gb_bfs_noalloc(p, p, p, p, limit + 1, 0, 0, p, None, None, None)
    assert rc == gb.INVALID_VALUE
    assert f"1..{limit}" in gb.last_error()
