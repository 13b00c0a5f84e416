"""The C ABI library loads and exports what include/lf.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "lf.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"LF_API\s+[\w\s\*]*?\b(lf_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as lf

    return lf.load_library()


def test_header_declarations_parsed():
    names = _declared()
    assert "lf_render" in names and "lf_load_views" in names and len(names) >= 11


def test_every_declared_symbol_exported(lib):
    import paper_1810_08860_gb300 as lf

    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(lf.EXPORTS) == _declared()


def test_host_only_entry_points(lib):
    import paper_1810_08860_gb300 as lf

    cfg = lf.Config()
    lib.lf_config_default(ctypes.byref(cfg))
    assert (cfg.tile_w, cfg.tile_h, cfg.max_eyes) == (16, 16, 2)
    assert abs(cfg.z_near - 0.1) < 1e-7 and cfg.tri_capacity > 0
    assert lib.lf_status_string(0) == b"LF_OK"
    assert lib.lf_status_string(7) == b"LF_ERR_CAPACITY"
    # argument checks that run before any CUDA call
    out = ctypes.c_void_p()
    bad = lf.Config()
    lib.lf_config_default(ctypes.byref(bad))
    bad.tile_w, bad.tile_h = 12, 12
    assert lib.lf_create(0, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad.tile_w, bad.tile_h = 16, 16
    bad.max_eyes = 1000
    assert lib.lf_create(0, ctypes.byref(bad), ctypes.byref(out)) == 1
    assert lib.lf_create(0, None, None) == 1
    lib.lf_destroy(None)
    assert lib.lf_get_stats(None, None) == 1
    assert lib.lf_last_error(None) == b""


def test_struct_sizes_match_header(lib):
    import paper_1810_08860_gb300 as lf

    assert ctypes.sizeof(lf.Pose) == 96
    assert ctypes.sizeof(lf.Intrinsics) == 40
    assert ctypes.sizeof(lf.Config) == 40
    assert ctypes.sizeof(lf.Stats) == 48
    assert ctypes.sizeof(lf.FragRecord) == 24
    assert lf.FRAG_RECORD_DTYPE.itemsize == 24
