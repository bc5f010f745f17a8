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


@pytest.mark.parametrize("bad", [
    dict(nr=1), dict(r_min=0.0), dict(r_max=0.5), dict(r_map=2), dict(th_map=2), dict(n_filt=17),
    dict(absorb_cells=64), dict(vacuum=6), dict(precision=2), dict(pusher=2), dict(tile_shape=3),
    dict(inject=3), dict(inject=1, f_inj=1.5), dict(inject=1, f_inj=0.0), dict(inject=2, f_inj=0.5, inject_q=0.0),
    dict(inject=2, f_inj=0.5, inject_q=float("inf")), dict(inject_smooth=65), dict(inject_smooth=-1),
    dict(flux_quantum=-1.0),
])
def test_descriptor_validation_rejects_bad_values(bad):
    """pic_init_grid checks the descriptor before any device work, so a bad
    value is refused with PIC_EINVAL on any machine."""
    from paper_1407_1810_gb300 import build, picsar as P

    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    kw = dict(nr=64, nth=64, r_min=1.0, r_max=10.0, r_map="log", th_map="linear", dt=0.01, n_filt=0,
              absorb_cells=8, absorb_profile="linear", vacuum="monopole", b0=1.0, precision="fp64", pusher="vay")
    kw.update(bad)
    with pytest.raises(P.PicError) as e:
        P.Simulation(P.make_desc(**kw))
    assert e.value.code == P.PIC_EINVAL


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c", "c11"), ("c++", "c++17")])
def test_header_compiles_as_plain_c_and_cpp(lang, std):
    """include/picsar.h is the boundary for C callers: it must compile on its
    own, pedantically, without CUDA or torch headers."""
    import shutil
    import subprocess

    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    r = subprocess.run([cc, f"-std={std}", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", lang,
                        os.path.join(ROOT, "include", "picsar.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("nslabs,rows,over", [
    (16, None, {}),              # slabs of 4 rows are narrower than their halos (2 (n_filt + 2) + 2 rows)
    (2, [0, 40, 60], {}),        # the rows do not end at nr
    (2, [0, 56, 64], {}),        # the lossy layer (8 cells) does not fit in the last slab
    (3, [0, 30, 20, 64], {}),    # the rows do not increase
    (0, None, {}),
])
def test_slab_descriptor_and_rows_are_checked(nslabs, rows, over):
    """pic_slabs_init checks the grid, the slab rows and the path before any
    device work: refused with PIC_EINVAL on any machine."""
    from paper_1407_1810_gb300 import build, picsar as P

    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    kw = dict(nr=64, nth=40, r_min=1.0, r_max=10.0, r_map="log", th_map="linear", dt=0.01, n_filt=0,
              absorb_cells=8, absorb_profile="linear", vacuum="monopole", b0=1.0, precision="fp64", pusher="vay")
    kw.update(over)
    with pytest.raises(P.PicError) as e:
        P.Slabs(P.make_desc(**kw), nslabs, rows)
    assert e.value.code == P.PIC_EINVAL
