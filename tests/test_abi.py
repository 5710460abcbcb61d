"""The C ABI library builds, loads and exports every entry point include/frsg.h declares.

Runs without a GPU: nvcc cross-compiles for sm_103a and ctypes only resolves symbols (no
compute call is made).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "frsg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fr_sg_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_05946_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["fr_sg_init", "fr_sg_destroy", "fr_sg_set_initial_nodal", "fr_sg_rhs", "fr_sg_rk_step",
                     "fr_sg_filter", "fr_sg_limit", "fr_sg_moments", "fr_sg_cfl_dt"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2112_05946_gb300 import frsg
    assert sorted(frsg.exported_names()) == _declared()


def test_config_struct_size_matches_header_layout(lib):
    """sizeof(frsg_config) as the binding lays it out must be what fr_sg_init checks."""
    from paper_2112_05946_gb300 import frsg
    c = frsg.make_config()
    assert c.struct_size == ctypes.sizeof(frsg.Config)
    # fr_sg_init rejects a wrong struct_size before touching the GPU
    bad = frsg.make_config()
    bad.struct_size = 7
    h = ctypes.c_void_p()
    fn = lib.fr_sg_init
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(frsg.Config), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    assert fn(ctypes.byref(bad), None, ctypes.byref(h)) == frsg.E_INVAL
    assert not h.value


def test_tune_cache_file_roundtrip(tmp_path):
    """The autotuner cache file is host-only: save, load, and reject malformed files."""
    from paper_2112_05946_gb300 import frsg
    frsg.load_library()
    p = tmp_path / "tune.txt"
    frsg.tune_cache_save(str(p))
    assert p.read_text().startswith("frsg-tune 1")
    p.write_text("frsg-tune 1\n1 3 8 16 1 1 1024 1 1 0 0 1 4\n1 3 8 16 1 1 1024 3 1 0 0 3 7\n")
    frsg.tune_cache_load(str(p))
    frsg.tune_cache_save(str(p))
    assert "1 3 8 16 1 1 1024 1 1 0 0 1 4" in p.read_text()
    assert "1 3 8 16 1 1 1024 3 1 0 0 3 7" in p.read_text()
    bad = tmp_path / "bad.txt"
    bad.write_text("frsg-tune 1\n1 2 3\n")
    with pytest.raises(frsg.FrsgError):
        frsg.tune_cache_load(str(bad))
    bad.write_text("frsg-tune 1\n1 3 8 16 1 1 1024 3 1 0 0 4 7\n")   # no layout 4
    with pytest.raises(frsg.FrsgError):
        frsg.tune_cache_load(str(bad))
    with pytest.raises(frsg.FrsgError):
        frsg.tune_cache_load(str(tmp_path / "missing.txt"))


def test_peak_library_exports_its_header():
    """libfrsg_peak.so (the FMA microbenchmark) exports what include/frsg_peak.h declares."""
    from paper_2112_05946_gb300 import build
    build.build()
    txt = open(os.path.join(ROOT, "include", "frsg_peak.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = sorted(set(re.findall(r"\b(frsg_[a-z0-9_]+)\s*\(", txt)))
    assert names == ["frsg_peak_fma"]
    lib = ctypes.CDLL(build.PEAK_OUT)
    for n in names:
        assert hasattr(lib, n), n
