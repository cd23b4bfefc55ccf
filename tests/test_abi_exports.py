"""The C-ABI library loads and exports every function include/btree.h
declares (no CUDA work is done: this runs on hosts without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "btree.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", txt, re.M)
    return sorted({n for n in names if n.startswith(("btree_", "sph_"))})


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("btree_build", "btree_find_neighbors", "btree_find_neighbors_density",
              "sph_density", "btree_free", "btree_strerror", "btree_status",
              "btree_get_info", "btree_export"):
        assert f in names


def test_library_exports_every_declared_symbol():
    from paper_1910_02639_gb300 import build_ext
    lib = ctypes.CDLL(build_ext.build())
    for name in _declared():
        assert hasattr(lib, name), name
    lib.btree_strerror.restype = ctypes.c_char_p
    assert lib.btree_strerror(0) == b"ok"
    assert lib.btree_strerror(-5).startswith(b"non-finite")


def test_argument_errors_need_no_device():
    """Invalid arguments are rejected before any CUDA call."""
    from paper_1910_02639_gb300 import build_ext
    lib = ctypes.CDLL(build_ext.build())
    out = ctypes.c_void_p(None)
    lib.btree_build.restype = ctypes.c_int
    vp = ctypes.c_void_p
    lib.btree_build.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, vp, vp, ctypes.POINTER(vp)]
    assert lib.btree_build(None, None, None, None, -1, 16, 0.5, 0.5, None, None,
                           ctypes.byref(out)) == -1
    assert lib.btree_build(None, None, None, None, 10, 16, 0.5, 0.5, None, None,
                           ctypes.byref(out)) == -1
    assert lib.btree_build(None, None, None, None, 0, 0, 0.5, 0.5, None, None,
                           ctypes.byref(out)) == -1
    assert lib.btree_build(None, None, None, None, 0, 16, float("nan"), 0.5, None, None,
                           ctypes.byref(out)) == -1
    lib.btree_find_neighbors.restype = ctypes.c_int
    lib.btree_find_neighbors.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    assert lib.btree_find_neighbors(None, 8, None, None, None) == -1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib
    import paper_1910_02639_gb300 as pkg
    monkeypatch.setattr(pkg, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    try:
        pkg._load()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("loading a missing library must raise")
    importlib.reload(pkg)
