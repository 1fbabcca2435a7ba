"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point include/vrc.h declares; struct layouts agree with the binding."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vrc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vrc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1111_6661_b300 import build
    build.build()
    return ctypes.CDLL(build.OUT)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1111_6661_b300 import _vrc
    assert set(declared_functions()) == set(_vrc.PROTOTYPES)


def test_struct_sizes_match_header():
    from paper_1111_6661_b300 import _vrc
    # sizes implied by the C declarations on x86-64
    assert ctypes.sizeof(_vrc.vrc_config) == 24
    assert ctypes.sizeof(_vrc.vrc_stats) == 48
    assert ctypes.sizeof(_vrc.vrc_camera) == 48
    assert ctypes.sizeof(_vrc.vrc_raycfg) == 40
    assert ctypes.sizeof(_vrc.vrc_tuning) == 48
    assert ctypes.sizeof(_vrc.vrc_request) == 4216
    assert ctypes.sizeof(_vrc.vrc_result) == 96


def test_status_strings_and_no_device_error(lib):
    from paper_1111_6661_b300 import _vrc
    L = _vrc.load()
    assert L.vrc_status_str(0) == b"ok"
    assert L.vrc_status_str(-2).startswith(b"out of memory")
    # null arguments are rejected before any CUDA call
    assert L.vrc_create(None, None) == -1
    assert L.vrc_destroy(None) == -1
    assert L.vrc_composite(None, None, None, None, 0, 0, None) == -1


def test_binding_has_no_cpu_fallback(tmp_path):
    from paper_1111_6661_b300 import _vrc
    old = _vrc._lib
    try:
        _vrc._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            _vrc.load(str(tmp_path / "missing.so"))
    finally:
        _vrc._lib = old
