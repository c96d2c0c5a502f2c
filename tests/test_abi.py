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
