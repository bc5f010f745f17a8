"""The C-ABI library loads and exports every symbol include/picsar.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "picsar.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pic_init_grid", "pic_load_particles", "pic_step", "pic_get_fields", "pic_get_moments"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1407_1810_gb300 import build, picsar

    try:
        path = build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(picsar.EXPORTS) == set(declared_symbols())


def test_binding_structs_match_the_library():
    """The ctypes mirrors of pic_desc and pic_moments have the library's sizes."""
    from paper_1407_1810_gb300 import build, picsar

    try:
        path = build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    a, b = ctypes.c_int64(), ctypes.c_int64()
    lib.pic_struct_sizes(ctypes.byref(a), ctypes.byref(b))
    assert a.value == ctypes.sizeof(picsar.pic_desc)
    assert b.value == ctypes.sizeof(picsar.pic_moments)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1407_1810_gb300 import picsar

    monkeypatch.setattr(picsar, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(picsar, "_lib", None)
    with pytest.raises(ImportError):
        picsar.lib()
