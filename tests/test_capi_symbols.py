"""The C-ABI library builds, loads without a GPU and exports every declared call."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(roar_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2408_08933_gb300 import build_ext

    return build_ext.build()


def test_header_declares_the_search_boundary():
    names = _declared()
    for must in ("roar_index_create", "roar_index_destroy", "roar_search", "roar_search_host"):
        assert must in names


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath, mode=os.RTLD_NOW)   # also fails on any unresolved symbol
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_argument_checks_without_gpu(libpath):
    import paper_2408_08933_gb300 as pkg

    L = pkg.lib()
    assert L.roar_status_string(pkg.ROAR_EOVERFLOW) == b"visit cap reached"
    h = ctypes.c_void_p()
    # invalid arguments are rejected before any CUDA call
    assert L.roar_index_create(0, 64, 16, 0, None, None, 16, 64, 0, 0, ctypes.byref(h)) == pkg.ROAR_EINVAL
    assert L.roar_index_create(10, 62, 16, 0, None, None, 16, 64, 0, 0, ctypes.byref(h)) == pkg.ROAR_EINVAL
    assert L.roar_index_create(10, 64, 16, 0, None, None, 16, 64, 10, 0, ctypes.byref(h)) == pkg.ROAR_EINVAL
    assert L.roar_index_create(10, 64, 16, 0, None, None, 16, 129, 0, 0, ctypes.byref(h)) == pkg.ROAR_EINVAL
    assert L.roar_index_create(10, 64, 16, 1, None, None, 16, 64, 0, 0, ctypes.byref(h)) == pkg.ROAR_EINVAL
    assert L.roar_search(None, None, 1, 10, 10, None, None, None, None, None, None) == pkg.ROAR_EINVAL


def test_package_refuses_to_run_without_library(monkeypatch, tmp_path):
    import paper_2408_08933_gb300 as pkg
    from paper_2408_08933_gb300 import build_ext

    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(build_ext, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pkg.lib()
