"""The C ABI library loads and exports every entry point declared in include/az.h."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "az.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(az_[A-Za-z0-9_]+)\s*\(", src)
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


def test_mixed_precision_refuses_small_eps_h():
    # The mixed path's FP32 symbol inverse needs eps h >= 0.504; the tau0 =
    # 1e-10 shape parameter of Eq. constant_shapeparam (eps h = 0.327) is
    # refused before any device work (the mask pointer is never read).
    import ctypes as C
    import paper_2308_14490_gb300 as az
    import workloads as W
    n, T = 256, 1.5
    epsh = W.epsh_from_tau0(1e-10)
    g = az.make_grid(1, (n,), (2,), (T,))
    o = az.make_options(az.AZ_MIXED, 64, 1e-8, 0.0, 1, 1)
    h = C.c_void_p()
    dummy = (C.c_uint8 * 4)()
    eps = epsh / (2 * T / n)
    st = az._lib.az_setup(C.byref(g), dummy, None, 0, C.c_double(eps), az.AZ_GAUSS, C.c_double(1.0),
                          C.byref(o), None, C.byref(h))
    assert st == az.AZ_ERR_ARG and not h.value
    assert "AZ_FP64" in az.az_last_error()


def _c_struct_fields(src, name):
    """Member (type, name) pairs of `typedef struct { ... } name;` in the header."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src, flags=re.S)
    assert m, name
    out = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        mm = re.match(r"(.+?)\s*\b(\w+)\s*(\[\d+\])?$", decl)
        out.append((mm.group(1).replace(" ", ""), mm.group(2) + (mm.group(3) or "")))
    return out


def test_ctypes_structs_match_the_header():
    # the binding's ctypes mirrors of az_grid, az_options and az_info_t have
    # the header's members in the header's order, with the same widths
    import ctypes
    import paper_2308_14490_gb300 as az
    src = open(os.path.join(ROOT, "include", "az.h")).read()
    width = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
             "double": ctypes.c_double, "size_t": ctypes.c_size_t, "constdouble*": ctypes.c_void_p}
    for cname, py in (("az_grid", az.az_grid), ("az_options", az.az_options), ("az_info_t", az.az_info_t)):
        fields = _c_struct_fields(src, cname)
        assert [f[1].split("[")[0] for f in fields] == [f[0] for f in py._fields_], cname
        for (ctype, cfield), (pname, ptype) in zip(fields, py._fields_):
            n = int(cfield.split("[")[1][:-1]) if "[" in cfield else 1
            assert ctypes.sizeof(ptype) == n * ctypes.sizeof(width[ctype]), (cname, cfield)
