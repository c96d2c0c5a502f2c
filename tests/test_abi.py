"""The C-ABI library loads and exports every entry point include/cpals.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    import paper_2010_12056_gb300 as p
    return p.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "cpals.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cp_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "cp_init" in names and "cp_sweep_msdt" in names and "cp_free" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    import paper_2010_12056_gb300 as p
    assert sorted(p.exported_symbols()) == declared()


def test_invalid_arguments_rejected_before_device_use(lib):
    import paper_2010_12056_gb300 as p
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    fake = ctypes.c_void_p(16)          # never dereferenced: validation fails first
    assert lib.cp_init(ctypes.byref(h), 2, dims, 3, fake, 0, None, None, None) == 1  # N < 3
    assert lib.cp_init(ctypes.byref(h), 3, dims, 0, fake, 0, None, None, None) == 1  # R < 1
    assert lib.cp_init(ctypes.byref(h), 3, dims, 513, fake, 0, None, None, None) == 1
    assert lib.cp_init(ctypes.byref(h), 3, dims, 3, None, 0, None, None, None) == 1
    assert lib.cp_init(ctypes.byref(h), 3, dims, 3, fake, 3, None, None, None) == 1  # dtype
    bad = (ctypes.c_int64 * 3)(4, 0, 6)
    assert lib.cp_init(ctypes.byref(h), 3, bad, 3, fake, 0, None, None, None) == 1
    cfg = p.Config()
    lib.cp_config_default(ctypes.byref(cfg))
    assert cfg.prec == p.PREC["f16x3"] and abs(cfg.pp_eps - 0.1) < 1e-15
    cfg.prec = 9
    assert lib.cp_init(ctypes.byref(h), 3, dims, 3, fake, 0, None, ctypes.byref(cfg), None) == 1
    # NULL contexts
    assert lib.cp_sweep_dt(None, 1) == 1
    assert lib.cp_set_option(None, 2, 1) == 1
    assert lib.cp_fit(None, 0, None, None) == 1
    lib.cp_free(None)
    assert lib.cp_last_error(None) == b"null context"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2010_12056_gb300 as p
    monkeypatch.setattr(p, "_lib", None)
    monkeypatch.setattr(p, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        p.lib()


def _header_structs():
    """typedef struct { ... } name; of the header as [(field, ctypes type)] per name."""
    import ctypes as ct
    src = open(os.path.join(ROOT, "include", "cpals.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    ctype = {"int": ct.c_int, "int32_t": ct.c_int32, "int64_t": ct.c_int64, "uint64_t": ct.c_uint64,
             "double": ct.c_double, "float": ct.c_float}
    out = {}
    for m in re.finditer(r"typedef struct\s*\{([^}]*)\}\s*([a-z_]+)\s*;", src):
        fields = []
        for decl in m.group(1).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            t, rest = decl.split(None, 1)
            for name in rest.split(","):
                name = name.strip()
                arr = re.fullmatch(r"([a-z_0-9]+)\[(\d+)\]", name)
                fields.append((arr.group(1), ctype[t] * int(arr.group(2))) if arr else (name, ctype[t]))
        out[m.group(2)] = fields
    return src, out


def _same(a, b):
    """Two ctypes field lists with the same names, scalar types, array types and lengths."""
    if [n for n, _ in a] != [n for n, _ in b]:
        return False
    for (_, x), (_, y) in zip(a, b):
        if hasattr(x, "_length_") or hasattr(y, "_length_"):
            if getattr(x, "_length_", None) != getattr(y, "_length_", None) or x._type_ != y._type_:
                return False
        elif x != y:
            return False
    return True


def test_binding_options_and_structs_match_header():
    """The binding's option numbers and its mirrors of cp_config, cp_stats, cp_trace_rec
    and cp_probe_rec equal the header's: a field out of place would shift every value
    after it."""
    import paper_2010_12056_gb300 as p
    src, structs = _header_structs()
    opts = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"\bCP_OPT_([A-Z0-9_]+)\s*=\s*(\d+)", src)}
    assert opts == p.OPTIONS
    for cname, mirror in (("cp_config", p.Config), ("cp_stats", p.Stats), ("cp_trace_rec", p.TraceRec),
                          ("cp_probe_rec", p.ProbeRec)):
        assert _same(structs[cname], mirror._fields_), cname
