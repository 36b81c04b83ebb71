"""The C ABI library loads and exports every entry point declared in include/az.h."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "az.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(az_[A-Za-z_]+)\s*\(", src)
    return sorted(set(n for n in names if n not in ("az_handle",)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2308_14490_gb300 as az
    lib = ctypes.CDLL(az.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(az.EXPORTS) == declared


def test_host_side_errors_without_gpu():
    import paper_2308_14490_gb300 as az
    g = az.make_grid(1, (100,), (2,), (1.0,))   # not a power of two
    o = az.make_options()
    import ctypes as C
    b = C.c_size_t()
    st = az._lib.az_query_footprint(C.byref(g), 100, 0, C.byref(o), 2, C.byref(b))
    assert st == az.AZ_ERR_ARG
    assert "power" in az.az_last_error()
    g = az.make_grid(1, (1 << 20,), (2,), (1.0,))
    st = az._lib.az_query_footprint(C.byref(g), 1 << 20, 0, C.byref(o), 64, C.byref(b))
    assert st == az.AZ_OK and b.value > (1 << 20) * 24 * 4
