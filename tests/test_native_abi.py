"""CPU checks of the C ABI boundary: the library builds/loads and exports
every entry point declared in include/rverom.h; the Python binding declares
the same set; the product path refuses to run without the native library."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, 'include', 'rverom.h')


def declared():
    src = open(HEADER).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'^int\s+(\w+)\s*\(', src, flags=re.M)))


@pytest.fixture(scope='module')
def libpath():
    from paper_2306_02687_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_2306_02687_gb300 import build
        build.build()
    return _native.LIB_PATH


def test_header_declares_the_boundary():
    names = declared()
    for required in ('rve_rom_create', 'rve_rom_destroy', 'rve_rom_eval_batch', 'rve_rom_adjoint',
                     'macro_assemble', 'macro_gradient', 'macro_mesh_create'):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2306_02687_gb300 import _native
    assert sorted(_native.SIGNATURES) == declared()


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2306_02687_gb300 import _native
    monkeypatch.setattr(_native, '_lib', None)
    monkeypatch.setattr(_native, 'LIB_PATH', os.path.join(ROOT, 'no_such_dir', 'librverom.so'))
    with pytest.raises(RuntimeError, match='missing'):
        _native.lib()
