"""CPU-side checks of the boundary: the C-ABI library builds for sm_103a,
loads, and exports every function include/tsdf.h declares (no compute call
is made without a GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tsdf_[a-z_0-9]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1410_0925_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path_calls():
    names = _declared_functions()
    for n in ("tsdf_scene_create", "tsdf_integrate", "tsdf_read_blocks",
              "tsdf_load_blocks", "tsdf_lookup_blocks", "tsdf_status_string"):
        assert n in names


def test_library_exports_every_declared_function(lib):
    for n in _declared_functions():
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_every_declared_function():
    from paper_1410_0925_gb300 import tsdf
    assert set(_declared_functions()) <= set(tsdf.EXPORTED) | {"tsdf_status_string"}


def test_status_strings_without_gpu(lib):
    lib.tsdf_status_string.restype = ctypes.c_char_p
    assert lib.tsdf_status_string(0) == b"ok"
    assert b"pool" in lib.tsdf_status_string(-3)


def test_create_rejects_bad_descriptor_before_touching_the_device(lib):
    from paper_1410_0925_gb300.tsdf import SceneDesc
    lib.tsdf_scene_create.argtypes = [ctypes.POINTER(SceneDesc), ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    bad = SceneDesc(0.0, 0.02, 100, 10, 2, 64, 128, 0)
    assert lib.tsdf_scene_create(ctypes.byref(bad), None, ctypes.byref(h)) == -1
    bad = SceneDesc(0.01, 0.02, 100, 10, 2, 64, 128, 7)
    assert lib.tsdf_scene_create(ctypes.byref(bad), None, ctypes.byref(h)) == -1
    assert lib.tsdf_scene_create(None, None, ctypes.byref(h)) == -1
